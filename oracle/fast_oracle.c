/*
 * CPU oracle for the block-based FAST interest-point detector of the system
 * in Ye et al., arXiv 2202.13347 (Sec. 3.1.1: FAST corners, extracted per
 * block of a partition of the image so that the points spread evenly).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path
 * (the CUDA library under paper_2202_13347_gb300/) never calls it, and the
 * two share no code, headers or constants.
 *
 * The paper names the operator and the partitioning only.  The readings
 * taken where it is silent:
 *   segment test (FAST-9): the 16 pixels of the radius-3 Bresenham circle
 *   around p; p is a corner when 9 contiguous circle pixels are all brighter
 *   than I(p) + t or all darker than I(p) - t;
 *   score: the largest t for which p is still a corner, i.e. the largest
 *   over the 16 arcs of 9 of the arc's smallest difference I(c) - I(p)
 *   (brighter) or I(p) - I(c) (darker); p is a corner when score > t.  The
 *   differences are taken in FP32, as the image is stored, so the score is
 *   exactly the one the device computes;
 *   pixels closer than 3 to the border score 0;
 *   non-maximum suppression over 3 x 3: a corner survives when its score is
 *   at least every neighbour's and above the neighbours before it in raster
 *   order (the row above and the pixel to its left);
 *   block selection: grid_y x grid_x blocks (rows [by H / grid_y,
 *   (by + 1) H / grid_y), columns likewise); in each, among surviving corners
 *   at least `margin` from the image border, the highest score, ties to the
 *   smaller y, then the smaller x; (-1, -1) and score 0 when there is none.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* circle offsets (dx, dy), clockwise from the top */
static const int kCircle[16][2] = {{0, -3}, {1, -3}, {2, -2}, {3, -1}, {3, 0},  {3, 1},  {2, 2},  {1, 3},
                                   {0, 3},  {-1, 3}, {-2, 2}, {-3, 1}, {-3, 0}, {-3, -1}, {-2, -2}, {-1, -3}};

static float fo_score_px(const float* img, int W, int x, int y, float t) {
    const float c = img[(size_t)y * W + x];
    float d[16];
    for (int k = 0; k < 16; ++k) {
        const float v = img[(size_t)(y + kCircle[k][1]) * W + x + kCircle[k][0]];
        d[k] = v - c; /* FP32 difference, as stored */
    }
    float best = 0.0f;
    int first = 1;
    for (int s = 0; s < 16; ++s) {
        float mb = d[s], md = -d[s];
        for (int j = 1; j < 9; ++j) {
            const float v = d[(s + j) & 15];
            if (v < mb) mb = v;
            if (-v < md) md = -v;
        }
        const float m = mb > md ? mb : md;
        if (first || m > best) best = m;
        first = 0;
    }
    return best > t ? best : 0.0f;
}

/* FAST score of every pixel (0 where p is no corner or within 3 of the border) */
void oracle_fast_score(const float* img, int H, int W, float t, float* score) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            score[(size_t)y * W + x] = (y >= 3 && y < H - 3 && x >= 3 && x < W - 3) ? fo_score_px(img, W, x, y, t) : 0.0f;
}

/* 1 when the corner at (x, y) survives 3 x 3 non-maximum suppression */
static int fo_nms(const float* s, int H, int W, int x, int y) {
    const float v = s[(size_t)y * W + x];
    if (!(v > 0.0f)) return 0;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            if (!dx && !dy) continue;
            const int yy = y + dy, xx = x + dx;
            if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
            const float u = s[(size_t)yy * W + xx];
            const int before = dy < 0 || (dy == 0 && dx < 0);
            if (before ? !(v > u) : !(v >= u)) return 0;
        }
    return 1;
}

/*
 * Block-based FAST: one point per block (x, y in points[2b], points[2b+1],
 * its score in scores[b]; b = by * grid_x + bx).  Returns the number of
 * blocks with a point, -1 on bad arguments.
 */
int oracle_fast_blocks(const float* img, int H, int W, float t, int grid_y, int grid_x, int margin, int32_t* points,
                       float* scores) {
    if (H < 1 || W < 1 || grid_y < 1 || grid_x < 1 || grid_y > H || grid_x > W || margin < 0) return -1;
    float* s = (float*)malloc(sizeof(float) * (size_t)H * W);
    if (!s) return -1;
    oracle_fast_score(img, H, W, t, s);
    int found = 0;
    for (int by = 0; by < grid_y; ++by)
        for (int bx = 0; bx < grid_x; ++bx) {
            const int y0 = (int)((long long)by * H / grid_y), y1 = (int)((long long)(by + 1) * H / grid_y);
            const int x0 = (int)((long long)bx * W / grid_x), x1 = (int)((long long)(bx + 1) * W / grid_x);
            int bxp = -1, byp = -1;
            float bs = 0.0f;
            for (int y = y0; y < y1; ++y)
                for (int x = x0; x < x1; ++x) {
                    if (y < margin || y >= H - margin || x < margin || x >= W - margin) continue;
                    if (!fo_nms(s, H, W, x, y)) continue;
                    const float v = s[(size_t)y * W + x];
                    if (bxp < 0 || v > bs) { /* raster order: the first of equal scores stays */
                        bs = v;
                        bxp = x;
                        byp = y;
                    }
                }
            const int b = by * grid_x + bx;
            points[2 * b] = bxp;
            points[2 * b + 1] = byp;
            scores[b] = bxp >= 0 ? bs : 0.0f;
            found += bxp >= 0;
        }
    free(s);
    return found;
}
