/*
 * FP64 CPU oracle for the SFOC descriptor and Fast-NCC_SFOC matching of
 * Ye et al., "A Robust Multimodal Remote Sensing Image Registration Method
 * and System Using Steerable Filters with First- and Second-order
 * Gradients" (arXiv 2202.13347), Sec. 2.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path
 * (the CUDA library under paper_2202_13347_gb300/) never calls it, and the
 * two share no code, headers or constants.
 *
 * Everything is plain and slow on purpose: kernels are sampled as full 2-D
 * arrays from the closed forms, filtering is direct 2-D convolution with
 * clamp-to-edge borders, NCC is Eq. 8 evaluated literally with two-pass
 * means, all in double precision.  OpenMP only splits independent pixels or
 * points across threads; it never changes an operation's order.
 *
 * Readings of points the paper leaves open:
 *   sigma is a standard deviation (Sec. 2.1 text after Eq. 1 vs Eq. 6 text);
 *   kernel radius K = ceil(3 sigma), taps sampled at integer offsets;
 *   the second-order x (y) kernel is made zero-sum along its derivative axis;
 *   second-order basis S^60 := G_yy * I, S^120 := G_xy * I in Eq. 7;
 *   |.| of every steered response, summed over scales per orientation;
 *   dilated Gaussian smoothing with sigma_d = 1.0 (first group) and 1.5
 *   (second group), radius ceil(3 sigma_d), rates {1,2,3}, results summed;
 *   sigma_d = 0 switches a group's smoothing off (D = F, the descriptor
 *   "without Gaussian convolution" that Sec. 2.1 compares in Fig. 3);
 *   per-pixel L2 normalisation of each group, v / (||v|| + eps);
 *   clamp-to-edge borders for every convolution;
 *   a window (template) is flat when its variance is <= 1e-6 * mnz: NCC := 0
 *   (FLAT_TEMPLATE); FP32 noise on a constant image stays near 1e-10 per value;
 *   argmax order (NCC desc, dy asc, dx asc); 3-point parabola per axis.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_OUT_OF_BOUNDS 1
#define OR_FLAT_TEMPLATE 2
#define OR_PEAK_ON_EDGE 3
#define OR_NAN 4

#define OR_ERR_ARG (-1)
#define OR_ERR_ROI (-2)
#define OR_ERR_OOM (-3)

static const double OR_PI = 3.14159265358979323846;

typedef struct {
    int n_scales;          /* number of first-order scales */
    double scales[8];      /* first-order Gaussian STDs, Table 2: 0.6, 0.8, 1.0 */
    double sigma2;         /* second-order STD, Table 2: 1.5 */
    int n_orient;          /* orientations theta_k = k*pi/n_orient, Sec. 2.1: 6 */
    int n_dil;             /* number of dilation rates, Sec. 2.1: 3 */
    int dil[4];            /* dilation rates, Sec. 2.1: 1, 2, 3 */
    double sigma_d1;       /* smoothing STD of the first-order group */
    double sigma_d2;       /* smoothing STD of the second-order group ("larger") */
    double eps;            /* normalisation floor */
    int rectify;           /* 1: |.| of every steered response */
    double radius_mult;    /* K = ceil(radius_mult * sigma) */
    int first_order_only;  /* 1: F-SFOC (first-order group only) */
} oracle_params;

typedef struct {
    int32_t dx, dy;        /* integer offset of the best match, search = p + d */
    double ncc;            /* NCC at the best offset */
    double sub_dx, sub_dy; /* offset refined by the per-axis parabola */
    int32_t status;        /* OR_* */
    double margin;         /* best minus second-best NCC (0 if undefined) */
} oracle_result;

int oracle_num_threads(void) {
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

int oracle_radius(double sigma, double mult) {
    return (int)ceil(mult * sigma - 1e-9);
}

int oracle_channels(const oracle_params* p) {
    return p->first_order_only ? p->n_orient : 2 * p->n_orient;
}

static inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ---------------------------------------------------------------------- */
/* Kernels, Eq. 1-5.  Arrays are (2K+1) x (2K+1), index [(y+K)(2K+1)+(x+K)]. */
/* ---------------------------------------------------------------------- */

/* Eq. 2 and Eq. 3: first-order Gaussian derivatives along x and y. */
void oracle_kernel_g1(double sigma, int K, double* gx, double* gy) {
    int n = 2 * K + 1;
    double s2 = sigma * sigma, s4 = s2 * s2;
    for (int y = -K; y <= K; ++y)
        for (int x = -K; x <= K; ++x) {
            double e = exp(-(x * x + y * y) / (2.0 * s2));
            gx[(y + K) * n + (x + K)] = -(double)x / (2.0 * OR_PI * s4) * e;
            gy[(y + K) * n + (x + K)] = -(double)y / (2.0 * OR_PI * s4) * e;
        }
}

/* Eq. 5: G_xx, G_yy and G_xy.  G_xx is then made zero-sum along x (and G_yy
 * along y) by subtracting, for each row (column), its mean over the 2K+1
 * taps, so a constant image gives exactly zero second-order response. */
void oracle_kernel_g2(double sigma, int K, double* gxx, double* gyy, double* gxy) {
    int n = 2 * K + 1;
    double s2 = sigma * sigma, s4 = s2 * s2, s6 = s4 * s2;
    for (int y = -K; y <= K; ++y)
        for (int x = -K; x <= K; ++x) {
            double e = exp(-(x * x + y * y) / (2.0 * s2));
            gxx[(y + K) * n + (x + K)] = -(1.0 / (2.0 * OR_PI * s4)) * (1.0 - x * x / s2) * e;
            gyy[(y + K) * n + (x + K)] = -(1.0 / (2.0 * OR_PI * s4)) * (1.0 - y * y / s2) * e;
            gxy[(y + K) * n + (x + K)] = ((double)x * y / (2.0 * OR_PI * s6)) * e;
        }
    for (int y = 0; y < n; ++y) {
        double m = 0.0;
        for (int x = 0; x < n; ++x) m += gxx[y * n + x];
        m /= n;
        for (int x = 0; x < n; ++x) gxx[y * n + x] -= m;
    }
    for (int x = 0; x < n; ++x) {
        double m = 0.0;
        for (int y = 0; y < n; ++y) m += gyy[y * n + x];
        m /= n;
        for (int y = 0; y < n; ++y) gyy[y * n + x] -= m;
    }
}

/* Dilated Gaussian of Sec. 2.1: 1-D taps g(t) = exp(-t^2/2sd^2)/sum over
 * |t| <= Kd, placed at spacing r in both axes.  Full 2-D array of side
 * 2 r Kd + 1 with zeros in the holes. */
void oracle_kernel_dilated(double sigma_d, int Kd, int r, double* w) {
    int n = 2 * r * Kd + 1;
    double g[64];
    double s = 0.0;
    for (int t = -Kd; t <= Kd; ++t) {
        g[t + Kd] = exp(-(double)t * t / (2.0 * sigma_d * sigma_d));
        s += g[t + Kd];
    }
    for (int t = 0; t < 2 * Kd + 1; ++t) g[t] /= s;
    for (int i = 0; i < n * n; ++i) w[i] = 0.0;
    for (int u = -Kd; u <= Kd; ++u)
        for (int t = -Kd; t <= Kd; ++t)
            w[(r * u + r * Kd) * n + (r * t + r * Kd)] = g[u + Kd] * g[t + Kd];
}

/* Direct 2-D convolution with clamp-to-edge at one pixel:
 * sum over taps q of k(q) * img(clamp(y - qy), clamp(x - qx)). */
static inline double conv_at(const double* img, int H, int W, const double* k, int K, int y, int x) {
    int n = 2 * K + 1;
    double acc = 0.0;
    for (int qy = -K; qy <= K; ++qy) {
        int yy = clampi(y - qy, 0, H - 1);
        const double* row = img + (size_t)yy * W;
        const double* kr = k + (size_t)(qy + K) * n;
        for (int qx = -K; qx <= K; ++qx) {
            double kv = kr[qx + K];
            if (kv == 0.0) continue;
            acc += kv * row[clampi(x - qx, 0, W - 1)];
        }
    }
    return acc;
}

void oracle_conv2d(const double* img, int H, int W, const double* k, int K, double* out) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) out[(size_t)y * W + x] = conv_at(img, H, W, k, K, y, x);
}

/* ---------------------------------------------------------------------- */
/* SFOC cube on a region of interest, Eq. 6-7 and the text that follows.   */
/* ---------------------------------------------------------------------- */

/* Same as conv_at but the image is a float32 input read at clamped full-image
 * coordinates. */
static inline double conv_at_f(const float* img, int H, int W, const double* k, int K, int y, int x) {
    int n = 2 * K + 1;
    double acc = 0.0;
    for (int qy = -K; qy <= K; ++qy) {
        int yy = clampi(y - qy, 0, H - 1);
        const float* row = img + (size_t)yy * W;
        const double* kr = k + (size_t)(qy + K) * n;
        for (int qx = -K; qx <= K; ++qx) acc += kr[qx + K] * (double)row[clampi(x - qx, 0, W - 1)];
    }
    return acc;
}

/*
 * Computes the SFOC cube of a float32 image (H x W, row-major) on the
 * rectangle [y0, y0+h) x [x0, x0+w), writing cube[c][h][w] (z channels:
 * first-order orientations then second-order orientations).
 * Returns 0 or a negative error.
 */
int oracle_sfoc_roi(const float* image, int H, int W, const oracle_params* p,
                    int y0, int x0, int h, int w, double* cube) {
    if (!image || !p || !cube || H <= 0 || W <= 0 || h <= 0 || w <= 0) return OR_ERR_ARG;
    if (y0 < 0 || x0 < 0 || y0 + h > H || x0 + w > W) return OR_ERR_ROI;
    if (p->n_scales < 1 || p->n_scales > 8 || p->n_orient < 1 || p->n_orient > 8) return OR_ERR_ARG;
    if (p->n_dil < 1 || p->n_dil > 4) return OR_ERR_ARG;
    if (!(p->sigma_d1 >= 0.0) || !(p->sigma_d2 >= 0.0)) return OR_ERR_ARG;
    const int no = p->n_orient;
    const int z = oracle_channels(p);
    const int ns = p->n_scales;

    /* kernels */
    int K1[8];
    double* g1x[8];
    double* g1y[8];
    for (int s = 0; s < ns; ++s) {
        K1[s] = oracle_radius(p->scales[s], p->radius_mult);
        int n = 2 * K1[s] + 1;
        g1x[s] = (double*)malloc(sizeof(double) * n * n);
        g1y[s] = (double*)malloc(sizeof(double) * n * n);
        oracle_kernel_g1(p->scales[s], K1[s], g1x[s], g1y[s]);
    }
    int K2 = oracle_radius(p->sigma2, p->radius_mult);
    int n2 = 2 * K2 + 1;
    double* g2xx = (double*)malloc(sizeof(double) * n2 * n2);
    double* g2yy = (double*)malloc(sizeof(double) * n2 * n2);
    double* g2xy = (double*)malloc(sizeof(double) * n2 * n2);
    oracle_kernel_g2(p->sigma2, K2, g2xx, g2yy, g2xy);

    int Kd[2] = {oracle_radius(p->sigma_d1, p->radius_mult), oracle_radius(p->sigma_d2, p->radius_mult)};
    double sd[2] = {p->sigma_d1, p->sigma_d2};
    double* wd[2][4];
    int wK[2][4];
    int reach = 0;
    for (int g = 0; g < 2; ++g)
        for (int r = 0; r < p->n_dil; ++r) {
            if (sd[g] == 0.0) { /* no smoothing: no kernel */
                wK[g][r] = 0;
                wd[g][r] = NULL;
                continue;
            }
            int rate = p->dil[r];
            wK[g][r] = rate * Kd[g];
            int n = 2 * wK[g][r] + 1;
            wd[g][r] = (double*)malloc(sizeof(double) * n * n);
            oracle_kernel_dilated(sd[g], Kd[g], rate, wd[g][r]);
            if (wK[g][r] > reach) reach = wK[g][r];
        }

    /* steered, rectified, scale-summed channels F_k on the ROI grown by the
     * smoothing reach (clamped to the image) */
    int ey0 = y0 - reach < 0 ? 0 : y0 - reach;
    int ex0 = x0 - reach < 0 ? 0 : x0 - reach;
    int ey1 = y0 + h + reach > H ? H : y0 + h + reach;
    int ex1 = x0 + w + reach > W ? W : x0 + w + reach;
    int eh = ey1 - ey0, ew = ex1 - ex0;
    double* F = (double*)malloc(sizeof(double) * (size_t)z * eh * ew);
    if (!F) return OR_ERR_OOM;

    double ct[8], st[8];
    for (int k = 0; k < no; ++k) {
        ct[k] = cos(k * OR_PI / no);
        st[k] = sin(k * OR_PI / no);
    }

#pragma omp parallel for schedule(dynamic, 4)
    for (int yy = 0; yy < eh; ++yy) {
        for (int xx = 0; xx < ew; ++xx) {
            int y = ey0 + yy, x = ex0 + xx;
            double Ix[8], Iy[8];
            for (int s = 0; s < ns; ++s) {
                Ix[s] = conv_at_f(image, H, W, g1x[s], K1[s], y, x);   /* Eq. 6, S^0 */
                Iy[s] = conv_at_f(image, H, W, g1y[s], K1[s], y, x);   /* Eq. 6, S^90 */
            }
            for (int k = 0; k < no; ++k) {
                double f = 0.0;
                for (int s = 0; s < ns; ++s) {
                    double v = ct[k] * Ix[s] + st[k] * Iy[s];            /* Eq. 6, S^theta */
                    f += p->rectify ? fabs(v) : v;
                }
                F[((size_t)k * eh + yy) * ew + xx] = f;
            }
            if (!p->first_order_only) {
                double Ixx = conv_at_f(image, H, W, g2xx, K2, y, x);   /* Eq. 7, S^0 */
                double Iyy = conv_at_f(image, H, W, g2yy, K2, y, x);   /* Eq. 7, S^60 (reading) */
                double Ixy = conv_at_f(image, H, W, g2xy, K2, y, x);   /* Eq. 7, S^120 (reading) */
                for (int k = 0; k < no; ++k) {
                    double v = ct[k] * ct[k] * Ixx + st[k] * st[k] * Iyy - 2.0 * st[k] * ct[k] * Ixy;
                    F[((size_t)(no + k) * eh + yy) * ew + xx] = p->rectify ? fabs(v) : v;
                }
            }
        }
    }

    /* parallel dilated Gaussian smoothing, summed over rates, then group-wise
     * normalisation and stacking */
#pragma omp parallel for schedule(dynamic, 4)
    for (int yy = 0; yy < h; ++yy) {
        double D[16];
        for (int xx = 0; xx < w; ++xx) {
            int y = y0 + yy, x = x0 + xx;
            for (int c = 0; c < z; ++c) {
                int g = c < no ? 0 : 1;
                const double* Fc = F + (size_t)c * eh * ew;
                if (sd[g] == 0.0) { /* smoothing off: the steered channel itself */
                    D[c] = Fc[(size_t)(y - ey0) * ew + (x - ex0)];
                    continue;
                }
                double acc = 0.0;
                for (int r = 0; r < p->n_dil; ++r) {
                    int K = wK[g][r], n = 2 * K + 1;
                    const double* k = wd[g][r];
                    for (int qy = -K; qy <= K; ++qy) {
                        int sy = clampi(y - qy, 0, H - 1) - ey0;
                        for (int qx = -K; qx <= K; ++qx) {
                            double kv = k[(qy + K) * n + (qx + K)];
                            if (kv == 0.0) continue;
                            int sx = clampi(x - qx, 0, W - 1) - ex0;
                            acc += kv * Fc[(size_t)sy * ew + sx];
                        }
                    }
                }
                D[c] = acc;
            }
            int ng = p->first_order_only ? 1 : 2;
            for (int g = 0; g < ng; ++g) {
                double n2s = 0.0;
                for (int k = 0; k < no; ++k) n2s += D[g * no + k] * D[g * no + k];
                double den = sqrt(n2s) + p->eps;
                for (int k = 0; k < no; ++k) {
                    /* NaN inputs stay NaN so matching can report them */
                    double v = (den != den) ? NAN : (den > 0.0 ? D[g * no + k] / den : 0.0);
                    cube[((size_t)(g * no + k) * h + yy) * w + xx] = v;
                }
            }
        }
    }

    free(F);
    for (int s = 0; s < ns; ++s) { free(g1x[s]); free(g1y[s]); }
    free(g2xx); free(g2yy); free(g2xy);
    for (int g = 0; g < 2; ++g)
        for (int r = 0; r < p->n_dil; ++r) free(wd[g][r]);
    return 0;
}

/* Complexity model, Eq. 17-19: multiplications of Fast-NCC (FFT + integral
 * images) over those of direct NCC for an m x n template in an M x N window. */
double oracle_complexity_ratio(int z, int m, int n, int M, int N) {
    double MNz = (double)M * N * z;
    double T1 = 4.0 * MNz * log2(MNz);                                   /* Eq. 17 */
    double T2 = 3.0 * m * n * (double)z * (M - m + 1) * (double)(N - n + 1); /* Eq. 18 */
    return T1 / T2;                                                       /* Eq. 19 */
}

/* ---------------------------------------------------------------------- */
/* Integral image, Eq. 14-16                                               */
/* ---------------------------------------------------------------------- */

/* Exclusive prefix P of size (H+1) x (W+1): P[y][x] = sum of g over rows
 * < y and columns < x, built with the column-sum / row recursion of Eq. 15. */
void oracle_integral(const double* g, int H, int W, double* P) {
    int W1 = W + 1;
    for (int x = 0; x <= W; ++x) P[x] = 0.0;
    for (int y = 1; y <= H; ++y) {
        P[(size_t)y * W1] = 0.0;
        double s = 0.0;
        for (int x = 1; x <= W; ++x) {
            s += g[(size_t)(y - 1) * W + (x - 1)];
            P[(size_t)y * W1 + x] = P[(size_t)(y - 1) * W1 + x] + s;
        }
    }
}

/* Eq. 16 with the exclusive layout: sum over [y0, y1) x [x0, x1). */
double oracle_rect_sum(const double* P, int W, int y0, int x0, int y1, int x1) {
    int W1 = W + 1;
    return P[(size_t)y1 * W1 + x1] - P[(size_t)y0 * W1 + x1] - P[(size_t)y1 * W1 + x0] + P[(size_t)y0 * W1 + x0];
}

/* ---------------------------------------------------------------------- */
/* NCC_SFOC by Eq. 8, argmax and sub-pixel                                  */
/* ---------------------------------------------------------------------- */

/* A cube stored for the rectangle [roi_y0, roi_y0+roi_h) x [roi_x0, ...) of
 * an image of size H x W, laid out [c][roi_h][roi_w]. */
typedef struct {
    const double* data;
    int z, H, W;
    int roi_y0, roi_x0, roi_h, roi_w;
} oracle_cube;

static inline int cube_has(const oracle_cube* c, int y0, int x0, int h, int w) {
    return y0 >= c->roi_y0 && x0 >= c->roi_x0 && y0 + h <= c->roi_y0 + c->roi_h && x0 + w <= c->roi_x0 + c->roi_w;
}

static inline double cube_at(const oracle_cube* c, int ch, int y, int x) {
    return c->data[((size_t)ch * c->roi_h + (y - c->roi_y0)) * c->roi_w + (x - c->roi_x0)];
}

/* Template window rows/cols before the centre (even m: [p - m/2, p + m/2 - 1]). */
int oracle_template_half(int m) { return (m % 2) ? (m - 1) / 2 : m / 2; }

/* Parabola through (-1, cm), (0, c0), (1, cp): vertex offset, or 0 when the
 * curvature is not negative; clamped to [-0.5, 0.5].  The paper has no
 * sub-pixel step; this is the separable 3-point reading applied per axis. */
double oracle_parabola(double cm, double c0, double cp) {
    double den = cm - 2.0 * c0 + cp;
    if (!(den < 0.0)) return 0.0;
    double d = (cm - cp) / (2.0 * den);
    if (d > 0.5) d = 0.5;
    if (d < -0.5) d = -0.5;
    return d;
}

/* Picks the best offset of an NCC map (rows dy = -R..R, cols dx = -R..R) with
 * the order (NCC desc, dy asc, dx asc); NaN entries are skipped and flagged.
 * The most similar position is the control point (Sec. 3.2.2); the paper
 * gives no tie rule, so ties go to the smallest dy, then dx. */
void oracle_pick(const double* map, int R, oracle_result* out) {
    int P1 = 2 * R + 1;
    int best = -1, has_nan = 0;
    double bv = 0.0;
    for (int i = 0; i < P1 * P1; ++i) {
        double v = map[i];
        if (v != v) { has_nan = 1; continue; }
        if (best < 0 || v > bv) { best = i; bv = v; }
    }
    out->margin = 0.0;
    if (best < 0) {
        out->dx = out->dy = 0; out->ncc = 0.0; out->sub_dx = out->sub_dy = 0.0; out->status = OR_NAN;
        return;
    }
    double second = -INFINITY;
    for (int i = 0; i < P1 * P1; ++i)
        if (i != best && map[i] == map[i] && map[i] > second) second = map[i];
    out->margin = isinf(second) ? 0.0 : bv - second;
    int iy = best / P1, ix = best % P1;
    out->dy = iy - R;
    out->dx = ix - R;
    out->ncc = bv;
    int edge = 0;
    double ddx = 0.0, ddy = 0.0;
    if (ix > 0 && ix < P1 - 1) ddx = oracle_parabola(map[iy * P1 + ix - 1], bv, map[iy * P1 + ix + 1]);
    else edge = 1;
    if (iy > 0 && iy < P1 - 1) ddy = oracle_parabola(map[(iy - 1) * P1 + ix], bv, map[(iy + 1) * P1 + ix]);
    else edge = 1;
    if (ddx != ddx) ddx = 0.0;
    if (ddy != ddy) ddy = 0.0;
    out->sub_dx = out->dx + ddx;
    out->sub_dy = out->dy + ddy;
    out->status = has_nan ? OR_NAN : (edge ? OR_PEAK_ON_EDGE : OR_OK);
}

/*
 * Matches each point p (sensed coordinates, (x, y) pairs): the template is
 * the sensed cube on rows p_y - h .. p_y - h + m - 1 (same for columns); the
 * candidate at offset d in [-R, R]^2 is the reference cube on the same
 * rectangle shifted by d.  NCC by Eq. 8 with the means over all m*m*z values.
 * maps (optional) receives n x (2R+1)^2 NCC values, rows dy, cols dx.
 */
int oracle_match(const oracle_cube* ref, const oracle_cube* sen, const int32_t* pts, int n, int m, int R,
                 oracle_result* res, double* maps) {
    if (!ref || !sen || !res || n < 0 || m < 1 || R < 0) return OR_ERR_ARG;
    if (ref->z != sen->z) return OR_ERR_ARG;
    const int z = ref->z;
    const int h = oracle_template_half(m);
    const int P1 = 2 * R + 1;
    const double N = (double)m * m * z;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < n; ++k) {
        oracle_result* o = &res[k];
        double* map = maps ? maps + (size_t)k * P1 * P1 : NULL;
        memset(o, 0, sizeof(*o));
        if (map) for (int i = 0; i < P1 * P1; ++i) map[i] = 0.0;
        int px = pts[2 * k], py = pts[2 * k + 1];
        int ty0 = py - h, tx0 = px - h;
        if (ty0 < 0 || tx0 < 0 || ty0 + m > sen->H || tx0 + m > sen->W ||
            ty0 - R < 0 || tx0 - R < 0 || ty0 + m + R > ref->H || tx0 + m + R > ref->W) {
            o->status = OR_OUT_OF_BOUNDS;
            continue;
        }
        if (!cube_has(sen, ty0, tx0, m, m) || !cube_has(ref, ty0 - R, tx0 - R, m + 2 * R, m + 2 * R)) {
#pragma omp atomic write
            err = OR_ERR_ROI;
            continue;
        }
        /* template mean and centred energy (two passes) */
        double tsum = 0.0;
        int tnan = 0;
        for (int c = 0; c < z; ++c)
            for (int i = 0; i < m; ++i)
                for (int j = 0; j < m; ++j) {
                    double v = cube_at(sen, c, ty0 + i, tx0 + j);
                    if (v != v) tnan = 1;
                    tsum += v;
                }
        if (tnan) { o->status = OR_NAN; continue; }
        double tbar = tsum / N;
        double vT = 0.0;
        for (int c = 0; c < z; ++c)
            for (int i = 0; i < m; ++i)
                for (int j = 0; j < m; ++j) {
                    double d = cube_at(sen, c, ty0 + i, tx0 + j) - tbar;
                    vT += d * d;
                }
        if (vT <= 1e-6 * N) { o->status = OR_FLAT_TEMPLATE; continue; }
        double* lmap = map ? map : (double*)malloc(sizeof(double) * P1 * P1);
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                double ssum = 0.0;
                for (int c = 0; c < z; ++c)
                    for (int i = 0; i < m; ++i)
                        for (int j = 0; j < m; ++j) ssum += cube_at(ref, c, ty0 + i + dy, tx0 + j + dx);
                double sbar = ssum / N;
                double num = 0.0, vS = 0.0;
                for (int c = 0; c < z; ++c)
                    for (int i = 0; i < m; ++i)
                        for (int j = 0; j < m; ++j) {
                            double ds = cube_at(ref, c, ty0 + i + dy, tx0 + j + dx) - sbar;
                            double dt = cube_at(sen, c, ty0 + i, tx0 + j) - tbar;
                            num += ds * dt;
                            vS += ds * ds;
                        }
                double v;
                if (vS != vS || num != num) v = NAN;
                else if (vS <= 1e-6 * N) v = 0.0;
                else v = num / sqrt(vS * vT);
                lmap[(dy + R) * P1 + (dx + R)] = v;
            }
        oracle_pick(lmap, R, o);
        if (!map) free(lmap);
    }
    return err;
}

/* ---------------------------------------------------------------------- */
/* Second path for tiny inputs: Eq. 9 with R_ST from a naive DFT (Eq. 13)   */
/* and R_S, R_SS from integral images (Eq. 14-16).                          */
/* ---------------------------------------------------------------------- */

/*
 * S: search window cube [z][M][M], T: template [z][m][m], M = m + 2R.
 * Writes the (2R+1)^2 NCC map.  The correlation uses a linear (zero-padded)
 * DFT of side L >= M: R_ST(d) = IDFT[ sum_c DFT(S_c) conj(DFT(T_c)) ](d).
 */
int oracle_ncc_eq9_dft(const double* S, const double* T, int z, int m, int R, int L, double* map) {
    int M = m + 2 * R;
    if (L < M || L > 64) return OR_ERR_ARG;
    int P1 = 2 * R + 1;
    double N = (double)m * m * z;
    size_t LL = (size_t)L * L;
    double* accr = (double*)calloc(LL, sizeof(double));
    double* acci = (double*)calloc(LL, sizeof(double));
    double* sr = (double*)malloc(LL * sizeof(double));
    double* si = (double*)malloc(LL * sizeof(double));
    double* tr = (double*)malloc(LL * sizeof(double));
    double* ti = (double*)malloc(LL * sizeof(double));
    for (int c = 0; c < z; ++c) {
        /* naive 2-D DFT of the zero-padded S_c and T_c */
        for (int u = 0; u < L; ++u)
            for (int v = 0; v < L; ++v) {
                double a = 0, b = 0, e = 0, f = 0;
                for (int y = 0; y < L; ++y)
                    for (int x = 0; x < L; ++x) {
                        double ang = -2.0 * OR_PI * ((double)u * y / L + (double)v * x / L);
                        double cs = cos(ang), sn = sin(ang);
                        double sv = (y < M && x < M) ? S[((size_t)c * M + y) * M + x] : 0.0;
                        double tv = (y < m && x < m) ? T[((size_t)c * m + y) * m + x] : 0.0;
                        a += sv * cs; b += sv * sn;
                        e += tv * cs; f += tv * sn;
                    }
                sr[u * L + v] = a; si[u * L + v] = b;
                tr[u * L + v] = e; ti[u * L + v] = f;
            }
        /* S * conj(T), summed over channels */
        for (size_t q = 0; q < LL; ++q) {
            accr[q] += sr[q] * tr[q] + si[q] * ti[q];
            acci[q] += si[q] * tr[q] - sr[q] * ti[q];
        }
    }
    /* integral images of the channel-summed S and S^2 planes */
    double* g1 = (double*)calloc((size_t)M * M, sizeof(double));
    double* g2 = (double*)calloc((size_t)M * M, sizeof(double));
    for (int c = 0; c < z; ++c)
        for (int i = 0; i < M * M; ++i) {
            double v = S[(size_t)c * M * M + i];
            g1[i] += v;
            g2[i] += v * v;
        }
    double* P1s = (double*)malloc(sizeof(double) * (M + 1) * (M + 1));
    double* P2s = (double*)malloc(sizeof(double) * (M + 1) * (M + 1));
    oracle_integral(g1, M, M, P1s);
    oracle_integral(g2, M, M, P2s);
    double RT = 0.0, RTT = 0.0;
    for (int i = 0; i < z * m * m; ++i) { RT += T[i]; RTT += T[i] * T[i]; }
    double vT = RTT - RT * RT / N;
    for (int dy = 0; dy < P1; ++dy)
        for (int dx = 0; dx < P1; ++dx) {
            /* inverse DFT at (dy, dx) */
            double re = 0.0;
            for (int u = 0; u < L; ++u)
                for (int v = 0; v < L; ++v) {
                    double ang = 2.0 * OR_PI * ((double)u * dy / L + (double)v * dx / L);
                    re += accr[u * L + v] * cos(ang) - acci[u * L + v] * sin(ang);
                }
            double RST = re / (double)LL;
            double RS = oracle_rect_sum(P1s, M, dy, dx, dy + m, dx + m);
            double RSS = oracle_rect_sum(P2s, M, dy, dx, dy + m, dx + m);
            double vS = RSS - RS * RS / N;
            double num = RST - RS * RT / N;
            map[dy * P1 + dx] = (vS <= 1e-6 * N) ? 0.0 : num / (sqrt(vS) * sqrt(vT));
        }
    free(accr); free(acci); free(sr); free(si); free(tr); free(ti);
    free(g1); free(g2); free(P1s); free(P2s);
    return 0;
}
