/*
 * FP64 CPU oracle for the weight-sharing kernel-prediction denoiser of
 * Fan, Wang, Huo, Bao, "Real-time Monte Carlo Denoising with Weight Sharing
 * Kernel Prediction Network" (EGSR 2021).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously-correct loops in double
 * precision.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load this file; the denoiser library never does, and nothing here
 * is shared with the CUDA path.
 *
 * Layout: every image is planar [C][H][W] (row-major, x fastest) in double.
 * Conv weights are [Cout][Cin][KS][KS] followed by the bias [Cout], layer
 * after layer, in one flat array (the same blob the library takes).
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *  - Sec. 5.1: the 10 CNN input channels are gamma tone-mapped radiance
 *    clamp(r,0,1)^(1/gamma), albedo as is, normal 0.5 n + 0.5 and depth
 *    (d - near)/(far - near).
 *  - Sec. 4.1: each inference block is one KSxKS conv (zero padding KS/2,
 *    cross-correlation) + ReLU; the last layer is a linear conv whose
 *    channels 0..M-1 are the importance maps (Eq. 2) for kernel sizes
 *    k_0..k_{M-1} and channels M..2M-1 the fusion logits (Sec. 4.2).
 *  - Eq. 3/4: the filtering window is clipped to the image (pixels outside
 *    the image take no part in the softmax or the sum).
 *  - Sec. 4.2: the filter acts on irradiance y = r / (a + eps); the fused
 *    result is multiplied back by (a + eps).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { long x0, y0, x1, y1; } rect_t; /* half-open [x0,x1) x [y0,y1) */

static long lmax(long a, long b) { return a > b ? a : b; }
static long lmin(long a, long b) { return a < b ? a : b; }

static rect_t dilate_clip(rect_t r, long d, long H, long W) {
    rect_t o = { lmax(r.x0 - d, 0), lmax(r.y0 - d, 0), lmin(r.x1 + d, W), lmin(r.y1 + d, H) };
    return o;
}
static long rw(rect_t r) { return r.x1 - r.x0; }
static long rh(rect_t r) { return r.y1 - r.y0; }

int wo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- Sec. 5.1: input assembly --------------------------------------------
 * Computes the 10 network input channels on rect r (full-image buffers in,
 * region buffer out: 10 x rh x rw). */
static void prep_region(const double* rad, const double* alb, const double* nrm,
                        const double* dep, long H, long W, double gamma,
                        double dnear, double dfar, rect_t r, double* x0) {
    long w = rw(r), h = rh(r);
    for (long y = r.y0; y < r.y1; ++y)
        for (long x = r.x0; x < r.x1; ++x) {
            long g = y * W + x, l = (y - r.y0) * w + (x - r.x0);
            for (int c = 0; c < 3; ++c) {
                double v = rad[c * H * W + g];
                if (v < 0.0) v = 0.0;
                if (v > 1.0) v = 1.0;
                x0[c * h * w + l] = pow(v, 1.0 / gamma);           /* LDR radiance */
                x0[(3 + c) * h * w + l] = alb[c * H * W + g];          /* albedo */
                x0[(6 + c) * h * w + l] = 0.5 * nrm[c * H * W + g] + 0.5; /* normal -> [0,1] */
            }
            x0[9 * h * w + l] = (dep[g] - dnear) / (dfar - dnear);   /* depth -> [0,1] */
        }
}

void wo_prep(const double* rad, const double* alb, const double* nrm, const double* dep,
             long H, long W, double gamma, double dnear, double dfar, double* x0) {
    rect_t r = { 0, 0, W, H };
    prep_region(rad, alb, nrm, dep, H, W, gamma, dnear, dfar, r, x0);
}

/* ---- Sec. 4.1: one KSxKS convolution (+ optional ReLU) --------------------
 * in: Cin planes covering rect ri; out: Cout planes covering rect ro.
 * Every input pixel that a ro-pixel touches and that lies inside the image
 * must lie in ri; pixels outside the image read as zero (zero padding). */
static void conv_region(const double* in, rect_t ri, int Cin, const double* wt,
                        const double* bias, int Cout, int KS, int relu,
                        double* out, rect_t ro, long H, long W) {
    const int pad = KS / 2;
    const long wi = rw(ri), hi = rh(ri), wo = rw(ro), ho = rh(ro);
#pragma omp parallel for collapse(2) schedule(static)
    for (int o = 0; o < Cout; ++o)
        for (long y = ro.y0; y < ro.y1; ++y)
            for (long x = ro.x0; x < ro.x1; ++x) {
                double s = bias[o];
                for (int c = 0; c < Cin; ++c)
                    for (int dy = 0; dy < KS; ++dy) {
                        long yy = y + dy - pad;
                        if (yy < 0 || yy >= H) continue;
                        for (int dx = 0; dx < KS; ++dx) {
                            long xx = x + dx - pad;
                            if (xx < 0 || xx >= W) continue;
                            s += wt[((long)(o * Cin + c) * KS + dy) * KS + dx] *
                                 in[((long)c * hi + (yy - ri.y0)) * wi + (xx - ri.x0)];
                        }
                    }
                if (relu && s < 0.0) s = 0.0;
                out[((long)o * ho + (y - ro.y0)) * wo + (x - ro.x0)] = s;
            }
}

void wo_conv2d(const double* x, int Cin, long H, long W, const double* wt, const double* bias,
               int Cout, int KS, int relu, double* y) {
    rect_t r = { 0, 0, W, H };
    conv_region(x, r, Cin, wt, bias, Cout, KS, relu, y, r, H, W);
}

/* ---- Eq. 3 + Eq. 4, explicit per-pixel kernel construction ---------------
 * For pixel p=(px,py): the window Omega_p is the k x k neighbourhood clipped
 * to the image; w_p(q) = exp(I(q)) / sum_{q' in Omega_p} exp(I(q')) (computed
 * with the window maximum subtracted, which cancels); R(p) = sum w_p(q) y(q).
 * z and y are planes over rect rz (which must contain the clipped window). */
static void kernel_weights_px(const double* z, rect_t rz, long H, long W, int k,
                              long px, long py, double* wout /* k*k, row-major */) {
    const int h = (k - 1) / 2;
    const long wz = rw(rz);
    double m = -INFINITY, den = 0.0;
    for (long qy = lmax(py - h, 0); qy <= lmin(py + h, H - 1); ++qy)
        for (long qx = lmax(px - h, 0); qx <= lmin(px + h, W - 1); ++qx) {
            double v = z[(qy - rz.y0) * wz + (qx - rz.x0)];
            if (v > m) m = v;
        }
    for (long qy = lmax(py - h, 0); qy <= lmin(py + h, H - 1); ++qy)
        for (long qx = lmax(px - h, 0); qx <= lmin(px + h, W - 1); ++qx)
            den += exp(z[(qy - rz.y0) * wz + (qx - rz.x0)] - m);
    for (int j = 0; j < k * k; ++j) wout[j] = 0.0;
    for (long qy = lmax(py - h, 0); qy <= lmin(py + h, H - 1); ++qy)
        for (long qx = lmax(px - h, 0); qx <= lmin(px + h, W - 1); ++qx)
            wout[(qy - py + h) * k + (qx - px + h)] =
                exp(z[(qy - rz.y0) * wz + (qx - rz.x0)] - m) / den;
}

static void filter_px(const double* z, const double* y, rect_t rz, long H, long W, int k,
                      long px, long py, double* wbuf, double R[3]) {
    const int h = (k - 1) / 2;
    const long wz = rw(rz), hz = rh(rz);
    kernel_weights_px(z, rz, H, W, k, px, py, wbuf);
    R[0] = R[1] = R[2] = 0.0;
    for (int dy = -h; dy <= h; ++dy)
        for (int dx = -h; dx <= h; ++dx) {
            double wq = wbuf[(dy + h) * k + (dx + h)];
            if (wq == 0.0) continue; /* outside the image (or underflow: adds 0 anyway) */
            long qy = py + dy, qx = px + dx;
            long l = (qy - rz.y0) * wz + (qx - rz.x0);
            for (int c = 0; c < 3; ++c) R[c] += wq * y[c * hz * wz + l];
        }
}

/* Kernel weights of one pixel, exported for invariant checks. */
void wo_kernel_weights(const double* z, long H, long W, int k, long px, long py, double* w) {
    rect_t r = { 0, 0, W, H };
    kernel_weights_px(z, r, H, W, k, px, py, w);
}

/* Eq. 3-4 over a whole image: R[3][H][W] from one importance map z[H][W]
 * and the irradiance y[3][H][W]. */
void wo_decode_explicit(const double* z, const double* y, long H, long W, int k, double* R) {
    rect_t r = { 0, 0, W, H };
#pragma omp parallel
    {
        double* wbuf = (double*)malloc(sizeof(double) * k * k);
#pragma omp for schedule(static)
        for (long py = 0; py < H; ++py)
            for (long px = 0; px < W; ++px) {
                double Rp[3];
                filter_px(z, y, r, H, W, k, px, py, wbuf, Rp);
                for (int c = 0; c < 3; ++c) R[(long)c * H * W + py * W + px] = Rp[c];
            }
        free(wbuf);
    }
}

/* Second, independent coding of Eq. 3-4: with E(q) = exp(I(q) - g) for the
 * global maximum g, R(p) = (sum_{Omega_p} E y) / (sum_{Omega_p} E), i.e. a
 * ratio of two window sums (numerator per colour channel, one denominator). */
void wo_decode_boxsum(const double* z, const double* y, long H, long W, int k, double* R) {
    const int h = (k - 1) / 2;
    const long n = H * W;
    double g = -INFINITY;
    for (long i = 0; i < n; ++i) if (z[i] > g) g = z[i];
    double* E = (double*)malloc(sizeof(double) * n);
    double* EY = (double*)malloc(sizeof(double) * 3 * n);
    for (long i = 0; i < n; ++i) {
        E[i] = exp(z[i] - g);
        for (int c = 0; c < 3; ++c) EY[c * n + i] = E[i] * y[c * n + i];
    }
#pragma omp parallel for schedule(static)
    for (long py = 0; py < H; ++py)
        for (long px = 0; px < W; ++px) {
            double D = 0.0, N[3] = { 0.0, 0.0, 0.0 };
            for (long qy = lmax(py - h, 0); qy <= lmin(py + h, H - 1); ++qy)
                for (long qx = lmax(px - h, 0); qx <= lmin(px + h, W - 1); ++qx) {
                    D += E[qy * W + qx];
                    for (int c = 0; c < 3; ++c) N[c] += EY[c * n + qy * W + qx];
                }
            for (int c = 0; c < 3; ++c) R[c * n + py * W + px] = N[c] / D;
        }
    free(E);
    free(EY);
}

/* ---- Eq. 5 + Sec. 4.2: fusion weights (softmax over the M logits of a
 * pixel), weighted average of the M filtered results, albedo re-modulation. */
static void fuse_px(int M, const double* alogit, const double* Rm /* M x 3 */,
                    const double a[3], double eps, double out[3]) {
    double m = -INFINITY, s = 0.0;
    for (int i = 0; i < M; ++i) if (alogit[i] > m) m = alogit[i];
    for (int i = 0; i < M; ++i) s += exp(alogit[i] - m);
    double acc[3] = { 0.0, 0.0, 0.0 };
    for (int i = 0; i < M; ++i) {
        double alpha = exp(alogit[i] - m) / s;
        for (int c = 0; c < 3; ++c) acc[c] += alpha * Rm[i * 3 + c];
    }
    for (int c = 0; c < 3; ++c) out[c] = (a[c] + eps) * acc[c];
}

/* Full-image Eq. 5: Rs[M][3][H][W], alpha_logits[M][H][W], albedo[3][H][W]. */
void wo_fuse(const double* Rs, const double* alogits, const double* alb, int M,
             long H, long W, double eps, double* out) {
    const long n = H * W;
    double* al = (double*)malloc(sizeof(double) * M);
    double* Rm = (double*)malloc(sizeof(double) * M * 3);
    for (long i = 0; i < n; ++i) {
        double a[3], o[3];
        for (int j = 0; j < M; ++j) {
            al[j] = alogits[j * n + i];
            for (int c = 0; c < 3; ++c) Rm[j * 3 + c] = Rs[((long)j * 3 + c) * n + i];
        }
        for (int c = 0; c < 3; ++c) a[c] = alb[c * n + i];
        fuse_px(M, al, Rm, a, eps, o);
        for (int c = 0; c < 3; ++c) out[c * n + i] = o[c];
    }
    free(al);
    free(Rm);
}

/* ---- ImportanceNet forward on a rectangle --------------------------------
 * Computes the 2M output channels (Eq. 2 importance maps, then the fusion
 * logits) on rect rz, running each conv layer only on the part of the image
 * that the next layer needs.  widths[0..n_layers] (widths[0] == 10). */
static void logits_region(const double* rad, const double* alb, const double* nrm,
                          const double* dep, long H, long W, int n_layers, const int* widths,
                          int KS, const double* weights, double gamma, double dnear,
                          double dfar, rect_t rz, double* zout) {
    const int pad = KS / 2;
    rect_t* rr = (rect_t*)malloc(sizeof(rect_t) * (n_layers + 1));
    rr[n_layers] = rz;
    for (int l = n_layers - 1; l >= 0; --l) rr[l] = dilate_clip(rr[l + 1], pad, H, W);
    double* cur = (double*)malloc(sizeof(double) * widths[0] * rw(rr[0]) * rh(rr[0]));
    prep_region(rad, alb, nrm, dep, H, W, gamma, dnear, dfar, rr[0], cur);
    const double* wp = weights;
    for (int l = 1; l <= n_layers; ++l) {
        int Cin = widths[l - 1], Cout = widths[l];
        const double* wt = wp;
        const double* b = wp + (long)Cout * Cin * KS * KS;
        wp = b + Cout;
        double* nxt = (l == n_layers) ? zout
                                      : (double*)malloc(sizeof(double) * Cout * rw(rr[l]) * rh(rr[l]));
        conv_region(cur, rr[l - 1], Cin, wt, b, Cout, KS, l < n_layers, nxt, rr[l], H, W);
        free(cur);
        cur = (l == n_layers) ? NULL : nxt;
    }
    free(rr);
}

/* Network output (2M channels) on rect [x0,x1) x [y0,y1): out is
 * widths[n_layers] x (y1-y0) x (x1-x0). */
void wo_logits_region(const double* rad, const double* alb, const double* nrm, const double* dep,
                      long H, long W, int n_layers, const int* widths, int KS,
                      const double* weights, double gamma, double dnear, double dfar,
                      long x0, long y0, long x1, long y1, double* zout) {
    rect_t r = { x0, y0, x1, y1 };
    logits_region(rad, alb, nrm, dep, H, W, n_layers, widths, KS, weights, gamma, dnear, dfar,
                  r, zout);
}

/* Reconstruction (Eq. 3-5, Sec. 4.2) of the pixels in rect ro from network
 * outputs z given on rect rz (rz must contain ro dilated by the largest
 * half-window, clipped to the image). */
static void reconstruct_region(const double* z, rect_t rz, const double* rad, const double* alb,
                               long H, long W, int M, const int* ks, double eps,
                               rect_t ro, double* out) {
    const long wz = rw(rz), hz = rh(rz), nz = wz * hz;
    const long wo = rw(ro), ho = rh(ro);
    int kmax = 1;
    for (int i = 0; i < M; ++i) if (ks[i] > kmax) kmax = ks[i];
    /* irradiance y = r / (a + eps) on rz (Sec. 4.2 demodulation) */
    double* y = (double*)malloc(sizeof(double) * 3 * nz);
    for (long qy = rz.y0; qy < rz.y1; ++qy)
        for (long qx = rz.x0; qx < rz.x1; ++qx)
            for (int c = 0; c < 3; ++c)
                y[c * nz + (qy - rz.y0) * wz + (qx - rz.x0)] =
                    rad[(long)c * H * W + qy * W + qx] / (alb[(long)c * H * W + qy * W + qx] + eps);
#pragma omp parallel
    {
        double* wbuf = (double*)malloc(sizeof(double) * kmax * kmax);
        double* Rm = (double*)malloc(sizeof(double) * M * 3);
        double* al = (double*)malloc(sizeof(double) * M);
#pragma omp for collapse(2) schedule(static)
        for (long py = ro.y0; py < ro.y1; ++py)
            for (long px = ro.x0; px < ro.x1; ++px) {
                long l = (py - rz.y0) * wz + (px - rz.x0);
                for (int i = 0; i < M; ++i) {
                    filter_px(z + (long)i * nz, y, rz, H, W, ks[i], px, py, wbuf, Rm + 3 * i);
                    al[i] = z[(long)(M + i) * nz + l];
                }
                double a[3], o[3];
                for (int c = 0; c < 3; ++c) a[c] = alb[(long)c * H * W + py * W + px];
                fuse_px(M, al, Rm, a, eps, o);
                for (int c = 0; c < 3; ++c) out[((long)c * ho + (py - ro.y0)) * wo + (px - ro.x0)] = o[c];
            }
        free(wbuf);
        free(Rm);
        free(al);
    }
    free(y);
}

/* The whole denoiser D_Theta(r, f) (Eq. 1-5) evaluated on the pixels of the
 * rect [x0,x1) x [y0,y1) of an H x W frame; out is 3 x (y1-y0) x (x1-x0).
 * The full frame, a band of rows or a single pixel all go through the same
 * loops; only the part of each layer that the rect depends on is computed. */
void wo_denoise_region(const double* rad, const double* alb, const double* nrm, const double* dep,
                       long H, long W, int n_layers, const int* widths, int KS,
                       const double* weights, int M, const int* ks, double eps, double gamma,
                       double dnear, double dfar, long x0, long y0, long x1, long y1,
                       double* out) {
    int kmax = 1;
    for (int i = 0; i < M; ++i) if (ks[i] > kmax) kmax = ks[i];
    rect_t ro = { x0, y0, x1, y1 };
    rect_t rz = dilate_clip(ro, (kmax - 1) / 2, H, W);
    double* z = (double*)malloc(sizeof(double) * widths[n_layers] * rw(rz) * rh(rz));
    logits_region(rad, alb, nrm, dep, H, W, n_layers, widths, KS, weights, gamma, dnear, dfar,
                  rz, z);
    reconstruct_region(z, rz, rad, alb, H, W, M, ks, eps, ro, out);
    free(z);
}

/* Reconstruction only (decode + fusion + re-modulation) over a full frame
 * from given network outputs z[2M][H][W]. */
void wo_reconstruct(const double* z, const double* rad, const double* alb, long H, long W,
                    int M, const int* ks, double eps, double* out) {
    rect_t r = { 0, 0, W, H };
    reconstruct_region(z, r, rad, alb, H, W, M, ks, eps, r, out);
}

/* ---- Backward of the reconstruction (chain rule through Eq. 3-5) ---------
 * G = dL/dout [3][H][W]; writes dz [2M][H][W].  Follows the forward steps in
 * reverse with the explicit per-pixel kernels:
 *   out_c = (a_c+eps) sum_i alpha_i R_ic,  alpha = softmax(z_{M..2M-1}),
 *   R_ic(p) = sum_{q in Omega_i(p)} w_p(q) y_c(q),  w_p = softmax over Omega_i(p) of z_i.
 * dL/dR_ic(p) = (a_c+eps) G_c alpha_i;  dL/dw_p(q) = sum_c dL/dR_ic(p) y_c(q);
 * softmax: dz_i(q) += w_p(q) (dL/dw_p(q) - sum_{q'} w_p(q') dL/dw_p(q'));
 * dL/dalpha_i = sum_c (a_c+eps) G_c R_ic;  dz_{M+i} = alpha_i (dalpha_i - sum_j alpha_j dalpha_j). */
void wo_reconstruct_bwd(const double* z, const double* rad, const double* alb, long H, long W,
                        int M, const int* ks, double eps, const double* G, double* dz) {
    const long n = H * W;
    int kmax = 1;
    for (int i = 0; i < M; ++i) if (ks[i] > kmax) kmax = ks[i];
    double* y = (double*)malloc(sizeof(double) * 3 * n);
    for (long j = 0; j < n; ++j)
        for (int c = 0; c < 3; ++c) y[c * n + j] = rad[c * n + j] / (alb[c * n + j] + eps);
    double* alpha = (double*)malloc(sizeof(double) * M * n);
    for (long j = 0; j < n; ++j) {
        double m = -INFINITY, s = 0.0;
        for (int i = 0; i < M; ++i) if (z[(M + i) * n + j] > m) m = z[(M + i) * n + j];
        for (int i = 0; i < M; ++i) s += exp(z[(M + i) * n + j] - m);
        for (int i = 0; i < M; ++i) alpha[i * n + j] = exp(z[(M + i) * n + j] - m) / s;
    }
    double* Rall = (double*)malloc(sizeof(double) * M * 3 * n);
    memset(dz, 0, sizeof(double) * 2 * M * n);
    rect_t full = { 0, 0, W, H };
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < M; ++i) { /* each size writes only its own dz_i plane */
        const int k = ks[i], h = (k - 1) / 2;
        double* wbuf = (double*)malloc(sizeof(double) * k * k);
        double* dw = (double*)malloc(sizeof(double) * k * k);
        for (long py = 0; py < H; ++py)
            for (long px = 0; px < W; ++px) {
                long p = py * W + px;
                double R[3];
                filter_px(z + (long)i * n, y, full, H, W, k, px, py, wbuf, R);
                for (int c = 0; c < 3; ++c) Rall[((long)i * 3 + c) * n + p] = R[c];
                double dR[3];
                for (int c = 0; c < 3; ++c) dR[c] = (alb[c * n + p] + eps) * G[c * n + p] * alpha[i * n + p];
                double dot = 0.0;
                for (int dy = -h; dy <= h; ++dy)
                    for (int dx = -h; dx <= h; ++dx) {
                        long qy = py + dy, qx = px + dx;
                        int j = (dy + h) * k + (dx + h);
                        dw[j] = 0.0;
                        if (qy < 0 || qy >= H || qx < 0 || qx >= W) continue;
                        for (int c = 0; c < 3; ++c) dw[j] += dR[c] * y[c * n + qy * W + qx];
                        dot += wbuf[j] * dw[j];
                    }
                for (int dy = -h; dy <= h; ++dy)
                    for (int dx = -h; dx <= h; ++dx) {
                        long qy = py + dy, qx = px + dx;
                        if (qy < 0 || qy >= H || qx < 0 || qx >= W) continue;
                        int j = (dy + h) * k + (dx + h);
                        dz[(long)i * n + qy * W + qx] += wbuf[j] * (dw[j] - dot);
                    }
            }
        free(wbuf);
        free(dw);
    }
    for (long p = 0; p < n; ++p) {
        double da[64], s = 0.0; /* M <= 64 */
        for (int i = 0; i < M; ++i) {
            da[i] = 0.0;
            for (int c = 0; c < 3; ++c) da[i] += (alb[c * n + p] + eps) * G[c * n + p] * Rall[((long)i * 3 + c) * n + p];
            s += alpha[i * n + p] * da[i];
        }
        for (int i = 0; i < M; ++i) dz[(long)(M + i) * n + p] = alpha[i * n + p] * (da[i] - s);
    }
    free(y);
    free(alpha);
    free(Rall);
}

/* ---- Backward of one conv layer (pre-activation gradient gy given) -------
 * y[o,p] = b[o] + sum_{c,dy,dx} W[o,c,dy,dx] x[c, p + (dy,dx) - pad]:
 *   gW[o,c,dy,dx] = sum_p gy[o,p] x[c, p + d - pad]   (zero outside the image)
 *   gb[o]         = sum_p gy[o,p]
 *   gx[c,q]       = sum_{o,dy,dx} W[o,c,dy,dx] gy[o, q - d + pad]   (gx may be NULL) */
void wo_conv2d_bwd(const double* x, int Cin, long H, long W, const double* wt, int Cout, int KS,
                   const double* gy, double* gx, double* gw, double* gb) {
    const int pad = KS / 2;
    const long n = H * W;
#pragma omp parallel for collapse(2) schedule(static)
    for (int o = 0; o < Cout; ++o)
        for (int c = 0; c < Cin; ++c)
            for (int dy = 0; dy < KS; ++dy)
                for (int dx = 0; dx < KS; ++dx) {
                    double s = 0.0;
                    for (long py = 0; py < H; ++py) {
                        long yy = py + dy - pad;
                        if (yy < 0 || yy >= H) continue;
                        for (long px = 0; px < W; ++px) {
                            long xx = px + dx - pad;
                            if (xx < 0 || xx >= W) continue;
                            s += gy[o * n + py * W + px] * x[c * n + yy * W + xx];
                        }
                    }
                    gw[((long)(o * Cin + c) * KS + dy) * KS + dx] = s;
                }
    for (int o = 0; o < Cout; ++o) {
        double s = 0.0;
        for (long p = 0; p < n; ++p) s += gy[o * n + p];
        gb[o] = s;
    }
    if (!gx) return;
#pragma omp parallel for collapse(2) schedule(static)
    for (int c = 0; c < Cin; ++c)
        for (long qy = 0; qy < H; ++qy)
            for (long qx = 0; qx < W; ++qx) {
                double s = 0.0;
                for (int o = 0; o < Cout; ++o)
                    for (int dy = 0; dy < KS; ++dy) {
                        long py = qy - dy + pad;
                        if (py < 0 || py >= H) continue;
                        for (int dx = 0; dx < KS; ++dx) {
                            long px = qx - dx + pad;
                            if (px < 0 || px >= W) continue;
                            s += wt[((long)(o * Cin + c) * KS + dy) * KS + dx] * gy[o * n + py * W + px];
                        }
                    }
                gx[c * n + qy * W + qx] = s;
            }
}
