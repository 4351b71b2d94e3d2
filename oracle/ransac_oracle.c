/*
 * FP64 CPU oracle for the outlier rejection step of Ye et al., arXiv
 * 2202.13347 (Sec. 3.2.3: RANSAC with a projective transformation over the
 * control points) and for the matching criteria of Sec. 4.1 (number of
 * correct matches, correct matching ratio, RMSE of Eq. 22).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path
 * (the CUDA library under paper_2202_13347_gb300/) never calls it, and the
 * two share no code, headers or constants.
 *
 * The paper names the method and the model only.  The readings taken where
 * it is silent:
 *   model: x' = (h0 x + h1 y + h2) / (h6 x + h7 y + 1),
 *          y' = (h3 x + h4 y + h5) / (h6 x + h7 y + 1)   (projective, 8 dof);
 *          affine: h6 = h7 = 0 (6 dof);
 *   coordinates are normalised before any solve (Hartley): the centroid of
 *   the valid source (destination) points moves to the origin and their mean
 *   distance from it scales to sqrt(2); models are solved there and mapped
 *   back to pixels;
 *   a hypothesis is the exact solution on a minimal sample (4 points, affine
 *   3) whose indices are given (the random draws are inputs); a sample whose
 *   system is singular (pivot below 1e-12) is skipped;
 *   score = number of valid points whose reprojection error
 *   || H(src) - dst || is at most tau pixels; the highest score wins, ties go
 *   to the lower hypothesis index;
 *   final model: least squares over the winner's inliers with the same two
 *   equations per point, the inliers recounted with it, `refits` times.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Hartley normalisation of the valid points: T = (s, cx, cy) for
 * p -> s (p - c), mean distance of s (p - c) from the origin = sqrt(2). */
static void rs_norm(const double* p, const unsigned char* valid, int n, double* T) {
    double cx = 0.0, cy = 0.0;
    int cnt = 0;
    for (int i = 0; i < n; ++i)
        if (!valid || valid[i]) {
            cx += p[2 * i];
            cy += p[2 * i + 1];
            ++cnt;
        }
    if (cnt == 0) {
        T[0] = 1.0; T[1] = 0.0; T[2] = 0.0;
        return;
    }
    cx /= cnt;
    cy /= cnt;
    double md = 0.0;
    for (int i = 0; i < n; ++i)
        if (!valid || valid[i]) md += hypot(p[2 * i] - cx, p[2 * i + 1] - cy);
    md /= cnt;
    T[0] = md > 0.0 ? sqrt(2.0) / md : 1.0;
    T[1] = cx;
    T[2] = cy;
}

/* the two linear equations of one correspondence in the unknowns h0..h7
 * (projective) or h0..h5 (affine) */
static int rs_rows(int projective, double x, double y, double xp, double yp, double* r1, double* r2, double* b1,
                   double* b2) {
    const int nu = projective ? 8 : 6;
    memset(r1, 0, sizeof(double) * 8);
    memset(r2, 0, sizeof(double) * 8);
    r1[0] = x; r1[1] = y; r1[2] = 1.0;
    r2[3] = x; r2[4] = y; r2[5] = 1.0;
    if (projective) {
        r1[6] = -x * xp; r1[7] = -y * xp;
        r2[6] = -x * yp; r2[7] = -y * yp;
    }
    *b1 = xp;
    *b2 = yp;
    return nu;
}

/* Gaussian elimination with partial pivoting on the n x n system A x = b
 * (A, b overwritten).  Returns 0 when a pivot falls below 1e-12. */
static int rs_solve(double* A, double* b, int n, double* x) {
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * n + c]) > fabs(A[p * n + c])) p = r;
        if (fabs(A[p * n + c]) < 1e-12) return 0;
        if (p != c) {
            for (int k = 0; k < n; ++k) {
                double t = A[c * n + k]; A[c * n + k] = A[p * n + k]; A[p * n + k] = t;
            }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            const double f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * x[k];
        x[r] = s / A[r * n + r];
    }
    return 1;
}

/* the pixel model H = Td^-1 Hn Ts, scaled so that H[8] = 1; 0 if H[8] ~ 0 */
static int rs_denorm(const double* h, int projective, const double* Ts, const double* Td, double* H) {
    double Hn[9] = {h[0], h[1], h[2], h[3], h[4], h[5], projective ? h[6] : 0.0, projective ? h[7] : 0.0, 1.0};
    const double S[9] = {Ts[0], 0.0, -Ts[0] * Ts[1], 0.0, Ts[0], -Ts[0] * Ts[2], 0.0, 0.0, 1.0};
    const double Di[9] = {1.0 / Td[0], 0.0, Td[1], 0.0, 1.0 / Td[0], Td[2], 0.0, 0.0, 1.0};
    double M[9], R[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Hn[i * 3 + k] * S[k * 3 + j];
            M[i * 3 + j] = s;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Di[i * 3 + k] * M[k * 3 + j];
            R[i * 3 + j] = s;
        }
    if (fabs(R[8]) < 1e-300) return 0;
    for (int i = 0; i < 9; ++i) H[i] = R[i] / R[8];
    return 1;
}

/* squared reprojection error of src -> dst under H (infinite when the point
 * maps to infinity) */
static double rs_err2(const double* H, const double* s, const double* d) {
    const double w = H[6] * s[0] + H[7] * s[1] + H[8];
    if (w == 0.0) return INFINITY;
    const double xp = (H[0] * s[0] + H[1] * s[1] + H[2]) / w;
    const double yp = (H[3] * s[0] + H[4] * s[1] + H[5]) / w;
    return (xp - d[0]) * (xp - d[0]) + (yp - d[1]) * (yp - d[1]);
}

static int rs_count(const double* H, const double* src, const double* dst, const unsigned char* valid, int n,
                    double tau2, unsigned char* mask) {
    int c = 0;
    for (int i = 0; i < n; ++i) {
        const int in = (!valid || valid[i]) && rs_err2(H, src + 2 * i, dst + 2 * i) <= tau2;
        if (mask) mask[i] = (unsigned char)in;
        c += in;
    }
    return c;
}

/* Exact model on the k points idx[0..k-1] (k = 4 projective, 3 affine), in
 * the normalised frames Ts, Td; pixel model in H.  Returns 0 when singular. */
static int rs_fit_minimal(int projective, const double* src, const double* dst, const int* idx, const double* Ts,
                          const double* Td, double* H) {
    const int k = projective ? 4 : 3, nu = projective ? 8 : 6;
    double A[64], b[8], h[8], r1[8], r2[8], b1, b2;
    for (int j = 0; j < k; ++j) {
        const int i = idx[j];
        const double x = Ts[0] * (src[2 * i] - Ts[1]), y = Ts[0] * (src[2 * i + 1] - Ts[2]);
        const double xp = Td[0] * (dst[2 * i] - Td[1]), yp = Td[0] * (dst[2 * i + 1] - Td[2]);
        rs_rows(projective, x, y, xp, yp, r1, r2, &b1, &b2);
        for (int c = 0; c < nu; ++c) {
            A[(2 * j) * nu + c] = r1[c];
            A[(2 * j + 1) * nu + c] = r2[c];
        }
        b[2 * j] = b1;
        b[2 * j + 1] = b2;
    }
    if (!rs_solve(A, b, nu, h)) return 0;
    return rs_denorm(h, projective, Ts, Td, H);
}

/* Least squares over the points with mask[i] set (normal equations). */
static int rs_fit_ls(int projective, const double* src, const double* dst, const unsigned char* mask, int n,
                     const double* Ts, const double* Td, double* H) {
    const int nu = projective ? 8 : 6;
    double M[64], v[8], h[8], r1[8], r2[8], b1, b2;
    memset(M, 0, sizeof(M));
    memset(v, 0, sizeof(v));
    for (int i = 0; i < n; ++i) {
        if (!mask[i]) continue;
        const double x = Ts[0] * (src[2 * i] - Ts[1]), y = Ts[0] * (src[2 * i + 1] - Ts[2]);
        const double xp = Td[0] * (dst[2 * i] - Td[1]), yp = Td[0] * (dst[2 * i + 1] - Td[2]);
        rs_rows(projective, x, y, xp, yp, r1, r2, &b1, &b2);
        for (int a = 0; a < nu; ++a) {
            for (int c = 0; c < nu; ++c) M[a * nu + c] += r1[a] * r1[c] + r2[a] * r2[c];
            v[a] += r1[a] * b1 + r2[a] * b2;
        }
    }
    if (!rs_solve(M, v, nu, h)) return 0;
    return rs_denorm(h, projective, Ts, Td, H);
}

/*
 * RANSAC (Sec. 3.2.3).  src, dst: n x 2 pixel coordinates (sensed, reference);
 * valid: n flags or NULL; samples: n_hyp x k point indices (k = 4, or 3 for
 * the affine model); tau: inlier radius in pixels.  Outputs: H (3 x 3 row
 * major, H[8] = 1), inlier mask (n), the per-hypothesis scores (n_hyp; -1 for
 * a singular sample), the winning hypothesis (-1 if none) and the final
 * inlier count.  Returns 0 on success, -1 on bad arguments.
 */
int oracle_ransac(const double* src, const double* dst, const unsigned char* valid, int n, int projective,
                  const int* samples, int n_hyp, double tau, int refits, double* H, unsigned char* inlier,
                  int* scores, int* best, int* n_inliers) {
    const int k = projective ? 4 : 3;
    if (n < 0 || n_hyp < 0 || tau < 0.0 || refits < 0) return -1;
    for (int h = 0; h < n_hyp * k; ++h)
        if (samples[h] < 0 || samples[h] >= n) return -1;
    double Ts[3], Td[3];
    rs_norm(src, valid, n, Ts);
    rs_norm(dst, valid, n, Td);
    const double tau2 = tau * tau;
    int bi = -1, bs = -1;
    double Hb[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    for (int h = 0; h < n_hyp; ++h) {
        double Hh[9];
        int sc = -1;
        if (rs_fit_minimal(projective, src, dst, samples + (size_t)h * k, Ts, Td, Hh))
            sc = rs_count(Hh, src, dst, valid, n, tau2, NULL);
        scores[h] = sc;
        if (sc > bs) {
            bs = sc;
            bi = h;
            memcpy(Hb, Hh, sizeof(Hb));
        }
    }
    *best = bi;
    if (bi < 0) {
        for (int i = 0; i < 9; ++i) H[i] = (i % 4 == 0) ? 1.0 : 0.0;
        memset(inlier, 0, (size_t)n);
        *n_inliers = 0;
        return 0;
    }
    int cnt = rs_count(Hb, src, dst, valid, n, tau2, inlier);
    for (int it = 0; it < refits; ++it) {
        double Hr[9];
        if (cnt < k || !rs_fit_ls(projective, src, dst, inlier, n, Ts, Td, Hr)) break;
        memcpy(Hb, Hr, sizeof(Hb));
        cnt = rs_count(Hb, src, dst, valid, n, tau2, inlier);
    }
    memcpy(H, Hb, sizeof(Hb));
    *n_inliers = cnt;
    return 0;
}

/* The exact model on one minimal sample (exposed for the pins). */
int oracle_ransac_fit(const double* src, const double* dst, const unsigned char* valid, int n, int projective,
                      const int* idx, double* H) {
    double Ts[3], Td[3];
    rs_norm(src, valid, n, Ts);
    rs_norm(dst, valid, n, Td);
    return rs_fit_minimal(projective, src, dst, idx, Ts, Td, H);
}

/*
 * Matching criteria of Sec. 4.1 against a reference model P: a match is
 * correct when || dst - P(src) || <= tau (1.5 pixels in the paper);
 * NCM = correct matches, CMR = NCM / all matches, RMSE (Eq. 22) over the
 * correct ones.  Returns NCM; CMR and RMSE are 0 without matches.
 */
int oracle_match_quality(const double* P, const double* src, const double* dst, const unsigned char* valid, int n,
                         double tau, double* cmr, double* rmse) {
    int total = 0, ncm = 0;
    double se = 0.0;
    for (int i = 0; i < n; ++i) {
        if (valid && !valid[i]) continue;
        ++total;
        const double e2 = rs_err2(P, src + 2 * i, dst + 2 * i);
        if (e2 <= tau * tau) {
            ++ncm;
            se += e2;
        }
    }
    *cmr = total ? (double)ncm / total : 0.0;
    *rmse = ncm ? sqrt(se / ncm) : 0.0;
    return ncm;
}

/*
 * Rectification (Sec. 3.2.3, last paragraph): the sensed image resampled
 * into the reference frame with the fitted model H (sensed -> reference):
 * output pixel (x, y) of an out_h x out_w image takes the sensed image at
 * (u, v) = H^-1 (x, y) by bilinear interpolation (Sec. 3.2.3 names it);
 * positions outside [0, W-1] x [0, H-1] take `fill`.  H^-1 is the adjugate
 * of H scaled by its last entry; the interpolation weights and the blend
 * are computed in double and the result rounded to float once.
 * Returns 0, or -1 when H is singular.
 */
int oracle_rectify(const float* img, int H, int W, const double* Hm, float fill, int out_h, int out_w, float* out) {
    const double a = Hm[0], b = Hm[1], c = Hm[2], d = Hm[3], e = Hm[4], f = Hm[5], g = Hm[6], h = Hm[7], i = Hm[8];
    double inv[9] = {e * i - f * h, c * h - b * i, b * f - c * e, f * g - d * i, a * i - c * g,
                     c * d - a * f, d * h - e * g, b * g - a * h, a * e - b * d};
    const double det = a * inv[0] + b * inv[3] + c * inv[6];
    if (det == 0.0 || inv[8] == 0.0) return -1;
    for (int k = 0; k < 9; ++k) inv[k] /= inv[8];
    for (int y = 0; y < out_h; ++y)
        for (int x = 0; x < out_w; ++x) {
            const double w = inv[6] * x + inv[7] * y + inv[8];
            float v = fill;
            if (w != 0.0) {
                const double u = (inv[0] * x + inv[1] * y + inv[2]) / w;
                const double t = (inv[3] * x + inv[4] * y + inv[5]) / w;
                if (u >= 0.0 && t >= 0.0 && u <= W - 1 && t <= H - 1) {
                    int u0 = (int)floor(u), t0 = (int)floor(t);
                    if (u0 > W - 2) u0 = W - 2 < 0 ? 0 : W - 2;
                    if (t0 > H - 2) t0 = H - 2 < 0 ? 0 : H - 2;
                    const int u1 = u0 + 1 < W ? u0 + 1 : u0, t1 = t0 + 1 < H ? t0 + 1 : t0;
                    const double fu = u - u0, ft = t - t0;
                    const double p00 = img[(size_t)t0 * W + u0], p01 = img[(size_t)t0 * W + u1];
                    const double p10 = img[(size_t)t1 * W + u0], p11 = img[(size_t)t1 * W + u1];
                    v = (float)((1.0 - ft) * ((1.0 - fu) * p00 + fu * p01) + ft * ((1.0 - fu) * p10 + fu * p11));
                }
            }
            out[(size_t)y * out_w + x] = v;
        }
    return 0;
}
