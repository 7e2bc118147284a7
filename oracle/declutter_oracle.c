/*
 * Plain CPU oracle for one de-cluttering iteration of Rave, Molchanov and
 * Linsen, "De-cluttering Scatterplots with Integral Images" (arXiv 2408.06513).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * Arithmetic: FP64 for every real-valued quantity; exact unsigned 64-bit
 * integers for sample counts and for the integral images of integer grids.
 * Every function follows the paper's definitions in the paper's order, with
 * no blocking, fusion or reordering beyond what the definition states.
 *
 * Conventions (readings of the paper, each listed in the design notes):
 *   - grid of resolution N = 2^k (Sec. 4.1); pixel (i, j): i = column (x),
 *     j = row (y, pointing down), origin top-left (Sec. 4.1); row-major [j][i];
 *   - pixel (i, j) sits at (x, y) = (i, j) / N (Sec. 3.2, below eq. (map)),
 *     or at (i + 1/2, j + 1/2) / N when pixel_center is set;
 *   - a sample splats to pixel (floor(x N), floor(y N)), clamped to the grid,
 *     after clamping the coordinates to [0, 1] (NaN counts as 0).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(i, j, n) ((size_t)(j) * (size_t)(n) + (size_t)(i))

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

static double clamp01(double v)
{
    if (!(v >= 0.0)) return 0.0; /* also NaN */
    if (v > 1.0) return 1.0;
    return v;
}

/* ------------------------------------------------------------------------ */
/* Step 1 (Sec. 4.1, Sec. 4.3 step 1): single-pixel accumulation.            */
/* counts[j][i] = number of samples whose clamped position falls in pixel    */
/* (i, j).                                                                   */
/* ------------------------------------------------------------------------ */
void orc_splat(const float *xy, int64_t n, int N, uint64_t *counts)
{
    memset(counts, 0, sizeof(uint64_t) * (size_t)N * (size_t)N);
    for (int64_t p = 0; p < n; ++p) {
        double x = clamp01((double)xy[2 * p]);
        double y = clamp01((double)xy[2 * p + 1]);
        int i = (int)floor(x * N);
        int j = (int)floor(y * N);
        if (i > N - 1) i = N - 1;
        if (j > N - 1) j = N - 1;
        counts[IDX(i, j, N)] += 1;
    }
}

/* ------------------------------------------------------------------------ */
/* Step 1 continued (Sec. 4.1, Sec. 4.4): discrete Gaussian smoothing.       */
/* Weights g_k proportional to exp(-k^2 / (2 sigma^2)) for |k| <= r,         */
/* normalised to sum 1; sigma <= 0 means r / 3.  Separable: one horizontal   */
/* and one vertical pass.  Border: half-sample symmetric reflection          */
/* (-1 -> 0, N -> N-1), which keeps constants and the total mass.            */
/* ------------------------------------------------------------------------ */
void orc_gauss_weights(int r, double sigma, double *g)
{
    if (sigma <= 0.0) sigma = r / 3.0;
    double s = 0.0;
    for (int k = -r; k <= r; ++k) {
        g[k + r] = exp(-(double)k * (double)k / (2.0 * sigma * sigma));
        s += g[k + r];
    }
    for (int k = 0; k <= 2 * r; ++k) g[k] /= s;
}

static int reflect_index(int k, int N)
{
    if (k < 0) return -1 - k;
    if (k >= N) return 2 * N - 1 - k;
    return k;
}

void orc_smooth(const double *in, int N, int r, double sigma, double *out)
{
    double *g = (double *)malloc(sizeof(double) * (size_t)(2 * r + 1));
    double *tmp = (double *)malloc(sizeof(double) * (size_t)N * (size_t)N);
    orc_gauss_weights(r, sigma, g);
    /* horizontal pass */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            double s = 0.0;
            for (int k = -r; k <= r; ++k) s += g[k + r] * in[IDX(reflect_index(i + k, N), j, N)];
            tmp[IDX(i, j, N)] = s;
        }
    /* vertical pass */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            double s = 0.0;
            for (int k = -r; k <= r; ++k) s += g[k + r] * tmp[IDX(i, reflect_index(j + k, N), N)];
            out[IDX(i, j, N)] = s;
        }
    free(tmp);
    free(g);
}

/* ------------------------------------------------------------------------ */
/* Step 2 (Sec. 3.1): the eight integral images of a real texture.           */
/*                                                                           */
/* Each InIm is a sum over a quadrant.  The axis-aligned ones are quadrants  */
/* of the (i, j) grid; the tilted ones are quadrants of the rotated lattice  */
/* u = i + j, v = i - j.  A quadrant sum is computed as a running sum along  */
/* one axis followed by a running sum along the other, each over a closed or */
/* open half-line exactly as the definitions print it.                       */
/* ------------------------------------------------------------------------ */

/* Running sum along x of a row-major H x W array:
 *   upper = 0: out[y][x] = sum over x' <= x (x' <  x when strict)
 *   upper = 1: out[y][x] = sum over x' >= x (x' >  x when strict)       */
static void halfline_x(const double *a, int W, int H, int upper, int strict, double *out)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        const double *ar = a + (size_t)y * W;
        double *orow = out + (size_t)y * W;
        double run = 0.0;
        if (!upper) {
            for (int x = 0; x < W; ++x) {
                if (strict) { orow[x] = run; run += ar[x]; }
                else        { run += ar[x]; orow[x] = run; }
            }
        } else {
            for (int x = W - 1; x >= 0; --x) {
                if (strict) { orow[x] = run; run += ar[x]; }
                else        { run += ar[x]; orow[x] = run; }
            }
        }
    }
}

/* Running sum along y, same conventions. */
static void halfline_y(const double *a, int W, int H, int upper, int strict, double *out)
{
#pragma omp parallel for schedule(static)
    for (int x = 0; x < W; ++x) {
        double run = 0.0;
        if (!upper) {
            for (int y = 0; y < H; ++y) {
                double v = a[(size_t)y * W + x];
                if (strict) { out[(size_t)y * W + x] = run; run += v; }
                else        { run += v; out[(size_t)y * W + x] = run; }
            }
        } else {
            for (int y = H - 1; y >= 0; --y) {
                double v = a[(size_t)y * W + x];
                if (strict) { out[(size_t)y * W + x] = run; run += v; }
                else        { run += v; out[(size_t)y * W + x] = run; }
            }
        }
    }
}

/* inims: 8 planes of N*N doubles, in the order
 *   alpha, beta, gamma, delta, alpha_t, beta_t, gamma_t, delta_t.
 *
 * Sec. 3.1 definitions:
 *   alpha  : i' <= i, j' <= j        beta   : i' <= i, j' >  j
 *   gamma  : i' >  i, j' >  j        delta  : i' >  i, j' <= j
 *   alpha_t: u' <= u, v' >= v        beta_t : u' <= u, v' <  v
 *   gamma_t: u' >  u, v' <  v        delta_t: u' >  u, v' >= v
 * with u = i + j and v = i - j.                                            */
void orc_inims(const double *d, int N, double *inims)
{
    size_t NN = (size_t)N * N;
    double *tmp = (double *)malloc(sizeof(double) * NN);

    /* axis-aligned: x = i, y = j */
    /*              (x upper, x strict), (y upper, y strict)  */
    const int ax[4][4] = {
        {0, 0, 0, 0}, /* alpha: x' <= x, y' <= y */
        {0, 0, 1, 1}, /* beta : x' <= x, y' >  y */
        {1, 1, 1, 1}, /* gamma: x' >  x, y' >  y */
        {1, 1, 0, 0}, /* delta: x' >  x, y' <= y */
    };
    for (int q = 0; q < 4; ++q) {
        halfline_x(d, N, N, ax[q][0], ax[q][1], tmp);
        halfline_y(tmp, N, N, ax[q][2], ax[q][3], inims + (size_t)q * NN);
    }

    /* tilted: rotated lattice with rows u = i + j in [0, 2N-2] and columns
     * s = v + N - 1 = i - j + N - 1 in [0, 2N-2]; cells that are not pixels
     * hold zero. */
    int M = 2 * N - 1;
    size_t MM = (size_t)M * M;
    double *rot = (double *)calloc(MM, sizeof(double));
    double *rtmp = (double *)malloc(sizeof(double) * MM);
    double *rout = (double *)malloc(sizeof(double) * MM);
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) rot[(size_t)(i + j) * M + (i - j + N - 1)] = d[IDX(i, j, N)];
    /* columns (x) of the lattice carry v, rows (y) carry u */
    const int tl[4][4] = {
        {1, 0, 0, 0}, /* alpha_t: v' >= v, u' <= u */
        {0, 1, 0, 0}, /* beta_t : v' <  v, u' <= u */
        {0, 1, 1, 1}, /* gamma_t: v' <  v, u' >  u */
        {1, 0, 1, 1}, /* delta_t: v' >= v, u' >  u */
    };
    for (int q = 0; q < 4; ++q) {
        halfline_x(rot, M, M, tl[q][0], tl[q][1], rtmp);
        halfline_y(rtmp, M, M, tl[q][2], tl[q][3], rout);
        double *dst = inims + (size_t)(4 + q) * NN;
        for (int j = 0; j < N; ++j)
            for (int i = 0; i < N; ++i) dst[IDX(i, j, N)] = rout[(size_t)(i + j) * M + (i - j + N - 1)];
    }
    free(rout);
    free(rtmp);
    free(rot);
    free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Exact integer integral images of a uint32 grid (Sec. 3.1): alpha by the   */
/* summed-area recurrence, alpha_t by the tilted recurrence of Lienhart et   */
/* al. on a grid padded by N columns on each side:                           */
/*   at(i,j) = at(i-1,j-1) + at(i+1,j-1) - at(i,j-2) + g(i,j) + g(i,j-1).    */
/* Unsigned wrap-around in the subtraction is exact because every final      */
/* value is a non-negative sum that fits 64 bits.                            */
/* ------------------------------------------------------------------------ */
void orc_sat_u64(const uint32_t *g, int N, uint64_t *alpha, uint64_t *alpha_t)
{
    for (int j = 0; j < N; ++j) {
        uint64_t rowsum = 0;
        for (int i = 0; i < N; ++i) {
            rowsum += g[IDX(i, j, N)];
            alpha[IDX(i, j, N)] = rowsum + (j > 0 ? alpha[IDX(i, j - 1, N)] : 0);
        }
    }
    int W = 3 * N; /* padded columns: real column i sits at i + N */
    uint64_t *rows = (uint64_t *)calloc((size_t)3 * W, sizeof(uint64_t)); /* rows j, j-1, j-2 */
    for (int j = 0; j < N; ++j) {
        uint64_t *cur = rows + (size_t)(j % 3) * W;
        uint64_t *p1 = rows + (size_t)((j + 2) % 3) * W; /* row j-1 */
        uint64_t *p2 = rows + (size_t)((j + 1) % 3) * W; /* row j-2 */
        for (int c = 0; c < W; ++c) {
            int i = c - N;
            uint64_t gij = (i >= 0 && i < N) ? g[IDX(i, j, N)] : 0;
            uint64_t gij1 = (j >= 1 && i >= 0 && i < N) ? g[IDX(i, j - 1, N)] : 0;
            uint64_t a = (j >= 1 && c >= 1) ? p1[c - 1] : 0;
            uint64_t b = (j >= 1 && c + 1 < W) ? p1[c + 1] : 0;
            uint64_t e = (j >= 2) ? p2[c] : 0;
            cur[c] = a + b - e + gij + gij1;
        }
        for (int i = 0; i < N; ++i) alpha_t[IDX(i, j, N)] = cur[i + N];
    }
    free(rows);
}

/* ------------------------------------------------------------------------ */
/* Eq. (map) with the anchor points q1..q4 printed below it (Sec. 3.2):      */
/*   t(x,y;d) = ( alpha q1 + beta q2 + gamma q3 + delta q4                   */
/*              + alpha_t (x,1) + beta_t (1,y) + gamma_t (x,0)               */
/*              + delta_t (0,y) ) / (2C)                                     */
/*   y <  x : q1 = (1, 1+y-x),   q3 = (x-y, 0)                               */
/*   y >= x : q1 = (1-y+x, 1),   q3 = (0, y-x)                               */
/*   x+y < 1: q2 = (x+y, 0),     q4 = (0, x+y)                               */
/*   x+y >= 1: q2 = (1, x+y-1),  q4 = (x+y-1, 1)                             */
/* C is the total of the texture.  Output t: N*N*2 doubles (x, y).           */
/* The tie tests are taken on the pixel indices, which is exact.             */
/* ------------------------------------------------------------------------ */
void orc_mapping(const double *inims, int N, int pixel_center, double *t)
{
    size_t NN = (size_t)N * N;
    const double *al = inims, *be = inims + NN, *ga = inims + 2 * NN, *de = inims + 3 * NN;
    const double *alt = inims + 4 * NN, *bet = inims + 5 * NN, *gat = inims + 6 * NN, *det = inims + 7 * NN;
    /* alpha at the last pixel covers the whole texture */
    double C = al[IDX(N - 1, N - 1, N)];
    double off = pixel_center ? 0.5 : 0.0;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            size_t k = IDX(i, j, N);
            double x = (i + off) / N, y = (j + off) / N;
            int lower = (j < i);                                         /* y < x   */
            int below1 = pixel_center ? (i + j + 1 < N) : (i + j < N); /* x+y < 1 */
            double q1x, q1y, q2x, q2y, q3x, q3y, q4x, q4y;
            if (lower) { q1x = 1.0; q1y = 1.0 + y - x; q3x = x - y; q3y = 0.0; }
            else       { q1x = 1.0 - y + x; q1y = 1.0; q3x = 0.0; q3y = y - x; }
            if (below1) { q2x = x + y; q2y = 0.0; q4x = 0.0; q4y = x + y; }
            else        { q2x = 1.0; q2y = x + y - 1.0; q4x = x + y - 1.0; q4y = 1.0; }
            double Xx = al[k] * q1x + be[k] * q2x + ga[k] * q3x + de[k] * q4x
                      + alt[k] * x + bet[k] * 1.0 + gat[k] * x + det[k] * 0.0;
            double Xy = al[k] * q1y + be[k] * q2y + ga[k] * q3y + de[k] * q4y
                      + alt[k] * 1.0 + bet[k] * y + gat[k] * 0.0 + det[k] * y;
            if (C > 0.0) {
                t[2 * k] = Xx / (2.0 * C);
                t[2 * k + 1] = Xy / (2.0 * C);
            } else {
                t[2 * k] = x;
                t[2 * k + 1] = y;
            }
        }
}

/* ------------------------------------------------------------------------ */
/* Eqs. (d0) and (map_res), Sec. 4.1-4.3: d = d_r + d0, then                 */
/*   D(x,y) = t(x,y;d) - t(x,y;d0)                                           */
/* (the sample update adds D to the position).  The defect t(.;d0) is the    */
/* mapping of the constant texture; a constant of 1 is used when d0 = 0,     */
/* since the mapping of a constant does not depend on its value.  When the   */
/* texture d is empty (C = 0) the displacement is zero.                      */
/* D: N*N*2 doubles, domain units.                                           */
/* ------------------------------------------------------------------------ */
void orc_displacement(const double *d_r, int N, double d0, int pixel_center, double *D)
{
    size_t NN = (size_t)N * N;
    double *d = (double *)malloc(sizeof(double) * NN);
    double *inims = (double *)malloc(sizeof(double) * 8 * NN);
    double *td = (double *)malloc(sizeof(double) * 2 * NN);
    double *t0 = (double *)malloc(sizeof(double) * 2 * NN);
    double C = 0.0;
    for (size_t k = 0; k < NN; ++k) { d[k] = d_r[k] + d0; C += d[k]; }
    orc_inims(d, N, inims);
    orc_mapping(inims, N, pixel_center, td);
    double c0 = d0 > 0.0 ? d0 : 1.0;
    for (size_t k = 0; k < NN; ++k) d[k] = c0;
    orc_inims(d, N, inims);
    orc_mapping(inims, N, pixel_center, t0);
    for (size_t k = 0; k < 2 * NN; ++k) D[k] = (C > 0.0) ? td[k] - t0[k] : 0.0;
    free(t0);
    free(td);
    free(inims);
    free(d);
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.2 / Sec. 4.3 step 3: bilinear interpolation of the per-pixel       */
/* displacement at each sample, then z' = z + D(z); all samples use the same */
/* field.  With p = x N (x N - 1/2 for pixel centres): i0 = floor(p),        */
/* f = p - i0, corner indices clamped to the grid (constant extension at the */
/* right and bottom border).  Optional clamp of z' to [0,1]^2.  The result   */
/* is rounded to float32, the storage type of the samples.                   */
/* ------------------------------------------------------------------------ */
void orc_advect(const float *xy, int64_t n, int N, const double *D, int pixel_center, int clamp,
                float *out)
{
    double off = pixel_center ? 0.5 : 0.0;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; ++p) {
        double x = (double)xy[2 * p], y = (double)xy[2 * p + 1];
        double px = x * N - off, py = y * N - off;
        double fx0 = floor(px), fy0 = floor(py);
        double f = px - fx0, h = py - fy0;
        long ix = (long)fx0, iy = (long)fy0;
        long i0 = ix < 0 ? 0 : (ix > N - 1 ? N - 1 : ix);
        long i1 = ix + 1 < 0 ? 0 : (ix + 1 > N - 1 ? N - 1 : ix + 1);
        long j0 = iy < 0 ? 0 : (iy > N - 1 ? N - 1 : iy);
        long j1 = iy + 1 < 0 ? 0 : (iy + 1 > N - 1 ? N - 1 : iy + 1);
        double dx = (1 - h) * ((1 - f) * D[2 * IDX(i0, j0, N)] + f * D[2 * IDX(i1, j0, N)])
                  + h * ((1 - f) * D[2 * IDX(i0, j1, N)] + f * D[2 * IDX(i1, j1, N)]);
        double dy = (1 - h) * ((1 - f) * D[2 * IDX(i0, j0, N) + 1] + f * D[2 * IDX(i1, j0, N) + 1])
                  + h * ((1 - f) * D[2 * IDX(i0, j1, N) + 1] + f * D[2 * IDX(i1, j1, N) + 1]);
        double nx = x + dx, ny = y + dy;
        if (clamp) { nx = clamp01(nx); ny = clamp01(ny); }
        out[2 * p] = (float)nx;
        out[2 * p + 1] = (float)ny;
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 6.2 quality measures.                                                */
/*  out[0]: standard deviation of the sample counts of 4x4-pixel bins about  */
/*          their mean (population std over the (N/4)^2 bins);               */
/*  out[1]: that std divided by the mean bin count;                          */
/*  out[2]: overplotting = (n - number of occupied pixels) / n.              */
/* ------------------------------------------------------------------------ */
void orc_quality(const uint64_t *counts, int N, double *out)
{
    int B = N / 4;
    double n = 0.0;
    long occupied = 0;
    for (size_t k = 0; k < (size_t)N * N; ++k) {
        n += (double)counts[k];
        occupied += counts[k] > 0;
    }
    double mean = n / ((double)B * B);
    double ss = 0.0;
    for (int bj = 0; bj < B; ++bj)
        for (int bi = 0; bi < B; ++bi) {
            double s = 0.0;
            for (int j = 4 * bj; j < 4 * bj + 4; ++j)
                for (int i = 4 * bi; i < 4 * bi + 4; ++i) s += (double)counts[IDX(i, j, N)];
            ss += (s - mean) * (s - mean);
        }
    double sd = sqrt(ss / ((double)B * B));
    out[0] = sd;
    out[1] = mean > 0 ? sd / mean : 0.0;
    out[2] = n > 0 ? (n - (double)occupied) / n : 0.0;
}
