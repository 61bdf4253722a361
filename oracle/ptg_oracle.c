/*
 * ptg_oracle.c -- plain, slow, FP64 CPU oracle for polynomial terrain noise
 * (Thorimbert & Chopard, "Polynomial methods for fast Procedural Terrain
 * Generation", arXiv:1610.03525).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path and never calls it.
 *
 * What it computes (each function cites the passage it follows):
 *   - a counter-based lattice hash (pcg3d / pcg4d, Jarzynski & Olano,
 *     "Hash Functions for GPU Rendering", JCGT 9(3), 2020) giving each lattice
 *     corner a value and a gradient in [-1, 1).  The paper fixes no hash and no
 *     published test vectors are at hand: parity unpinned for the hash's exact
 *     words (its pins are statistical: uniform, uncorrelated, avalanche);
 *   - the fixed-point sample -> (cell, fraction) map of every octave (Sec. 2.1
 *     unit cell, Sec. 4 octave frequencies);
 *   - the corner constraint system of Eq. (mixedderiv) / Eq. (polynomial),
 *     built row by row from the derivative definition and solved numerically
 *     with LU and partial pivoting (never from a closed form);
 *   - the cell polynomial, evaluated monomial by monomial;
 *   - the fractal (fBm) octave sum of Sec. 4, and the ridged multifractal
 *     sum the paper renders its mountains with (Sec. 5.1, Fig. render2);
 *   - Perlin's polynomial of Sec. 3.2 and an OpenSimplex-style simplex-lattice
 *     gradient noise summed by brute force over a superset of lattice vertices;
 *   - the map statistics of Sec. 5: coastline box counts (Sec. 5.3) and the
 *     frequency distributions of height and slope (Sec. 5.1).
 *
 * Readings of the paper that this file depends on (the paper is silent or
 * inconsistent on them):
 *   - "C1" is the solution of the D2M1N3 / D3M1N3 system whose mixed corner
 *     derivatives (the twist terms) are zero: the tensor-product cubic Hermite
 *     cell.  Unlike the particular solution printed in Sec. 3.1 it is C1
 *     across cell faces.  The printed solution is available as the
 *     PAPER_GAUGE method (its four extra rows fix c22 = c33 = c32 = c23 = 0).
 *   - "C2" uses M = 2 with per-variable degree 5 (Sec. 3.4 names degree 4,
 *     which cannot meet the edge boundary condition of Eq. (independance) with
 *     six constraints per edge); every second-order and higher mixed corner
 *     derivative is zero.
 *   - Corner values and gradients are uniform in [-1, 1): u -> (u >> 9) 2^-22 - 1.
 *     Gradients are scaled by the weight w of Sec. 4.
 *   - Octave i has amplitude p^i and frequency 2^i times the base lattice;
 *     N octaves means i = 0 .. N-1; no normalisation of the sum.
 *   - Sample j of an axis sits at base-lattice coordinate origin + j / spc,
 *     spc = size / cells; cell indices wrap modulo 2^32.
 *   - The zero-gradient model of Eq. (zg) is taken with the sign of the xy
 *     term that the Sec. 3.1 coefficients give (-xy), not the printed +xy.
 *   - Ridged noise (shown in Sec. 5.1, defined by reference only): Musgrave's
 *     ridged multifractal (Ebert et al., "Texturing and Modeling", ch. 16) with
 *     offset 1 and gain 2 -- octave i contributes p^i r_i, r_i = (1 - |h_i|)^2
 *     w_i, w_0 = 1, w_{i+1} = clamp(2 r_i, 0, 1); h_i the unit-amplitude octave.
 *   - OpenSimplex-style noise: stretch (1/sqrt(3) - 1)/2, squish
 *     (sqrt(3) - 1)/2, kernel (2 - r^2)^4 (g . d), hashed gradients, scale 1/8;
 *     in 3D stretch -1/6, squish 1/3, the same kernel and scale.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Methods                                                                   */
/* ------------------------------------------------------------------------ */
enum {
    PTGO_C1 = 1,          /* tensor cubic Hermite (D?M1N3, zero twist)      */
    PTGO_C2 = 2,          /* tensor quintic Hermite (D?M2N5)                 */
    PTGO_PAPER_GAUGE = 3, /* D2M1N3 with the printed c22=c33=c32=c23=0 gauge */
    PTGO_ZERO_GRAD = 4,   /* Eq. (zg), -xy reading, f = g = 0               */
    PTGO_PERLIN_S5 = 10,  /* Perlin's polynomial, Sec. 3.2, S5 blend         */
    PTGO_PERLIN_S3 = 11,  /* Perlin's polynomial, Sec. 3.2, S3 blend         */
    PTGO_OPENSIMPLEX = 12 /* simplex-lattice gradient noise (Sec. 1 / 5.1)   */
};

typedef struct {
    int32_t dims;         /* 2 or 3                                        */
    int32_t method;       /* one of the PTGO_* methods                      */
    int64_t size[3];      /* samples per axis                               */
    int64_t cells[3];     /* base-lattice cells per axis                    */
    int64_t origin[3];    /* base-lattice cell of sample 0 (integer)        */
    int32_t octaves;      /* N, octaves 0 .. N-1                            */
    int32_t ridged;       /* 1: ridged multifractal sum instead of fBm      */
    double persistence;   /* p: amplitude ratio between octaves             */
    double grad_weight;   /* w of Sec. 4                                    */
    uint32_t seed;        /* < 2^24                                         */
    uint32_t pad2;
    double frequency;     /* f of Sec. 4, frequency ratio between octaves;
                             0 or 2 = the exact dyadic map of ptgo_axis      */
} ptgo_desc;

/* ------------------------------------------------------------------------ */
/* Hash: pcg3d / pcg4d (Jarzynski & Olano 2020), written from the published */
/* description: one LCG step per lane, a round of cross-lane multiply-adds, */
/* a 16-bit xorshift, a second round of cross-lane multiply-adds.           */
/* ------------------------------------------------------------------------ */
void ptgo_pcg3d(const uint32_t in[3], uint32_t out[3])
{
    uint32_t x = in[0] * 1664525u + 1013904223u;
    uint32_t y = in[1] * 1664525u + 1013904223u;
    uint32_t z = in[2] * 1664525u + 1013904223u;
    x += y * z;
    y += z * x;
    z += x * y;
    x ^= x >> 16;
    y ^= y >> 16;
    z ^= z >> 16;
    x += y * z;
    y += z * x;
    z += x * y;
    out[0] = x;
    out[1] = y;
    out[2] = z;
}

void ptgo_pcg4d(const uint32_t in[4], uint32_t out[4])
{
    uint32_t x = in[0] * 1664525u + 1013904223u;
    uint32_t y = in[1] * 1664525u + 1013904223u;
    uint32_t z = in[2] * 1664525u + 1013904223u;
    uint32_t w = in[3] * 1664525u + 1013904223u;
    x += y * w;
    y += z * x;
    z += x * y;
    w += y * z;
    x ^= x >> 16;
    y ^= y >> 16;
    z ^= z >> 16;
    w ^= w >> 16;
    x += y * w;
    y += z * x;
    z += x * y;
    w += y * z;
    out[0] = x;
    out[1] = y;
    out[2] = z;
    out[3] = w;
}

/* Hash word -> uniform value in [-1, 1): keep the top 23 bits. */
double ptgo_unit(uint32_t u)
{
    return (double)(u >> 9) * (1.0 / 4194304.0) - 1.0;
}

/* Key of octave i of a field: the seed in the high 24 bits, i in the low 8. */
static uint32_t octave_key(uint32_t seed, int octave)
{
    return (seed << 8) | (uint32_t)octave;
}

/* Value and gradient of one lattice corner (Sec. 3.1: h_ij, f_ij, g_ij).
 * out[0] = value, out[1 .. dims] = gradient components (unweighted). */
void ptgo_corner(int dims, const uint32_t* cell, uint32_t seed, int octave, double* out)
{
    uint32_t key = octave_key(seed, octave);
    if (dims == 2) {
        uint32_t in[3] = {cell[0], cell[1], key}, h[3];
        ptgo_pcg3d(in, h);
        for (int k = 0; k < 3; ++k) out[k] = ptgo_unit(h[k]);
    } else {
        uint32_t in[4] = {cell[0], cell[1], cell[2], key}, h[4];
        ptgo_pcg4d(in, h);
        for (int k = 0; k < 4; ++k) out[k] = ptgo_unit(h[k]);
    }
}

/* ------------------------------------------------------------------------ */
/* Coordinates (Sec. 2.1 unit cell; Sec. 4 frequency 2^i per octave).        */
/* Sample j of an axis sits at base coordinate origin + j/spc; at octave i   */
/* its lattice coordinate is that value times 2^i.  The integer part is the  */
/* cell (mod 2^32), the rest the position t in [0, 1) inside the cell.       */
/* ------------------------------------------------------------------------ */
void ptgo_axis(int64_t origin, int64_t spc, int64_t j, int octave, uint32_t* cell, double* t)
{
    uint64_t q = (uint64_t)j << octave;               /* j * 2^i, < 2^62 */
    uint64_t whole = q / (uint64_t)spc;
    uint64_t rem = q % (uint64_t)spc;
    *cell = (uint32_t)((uint64_t)origin << octave) + (uint32_t)whole;
    *t = (double)rem / (double)spc;
}

/* Any frequency ratio f (Sec. 4: f_i proportional to f^i): the lattice      */
/* coordinate of sample j at octave i is (origin + j/spc) f^i, in double.     */
/* The cell is its floor (mod 2^32), t the rest.                             */
void ptgo_axis_freq(int64_t origin, int64_t spc, int64_t j, double f, int octave, uint32_t* cell, double* t)
{
    const double u = ((double)origin + (double)j / (double)spc) * pow(f, (double)octave);
    const double fl = floor(u);
    *cell = (uint32_t)(uint64_t)(int64_t)fl;
    *t = u - fl;
}

void ptgo_axis_freq_batch(int64_t origin, int64_t spc, const int64_t* j, int64_t n, double f, int octave,
                          uint32_t* cell, double* t)
{
    for (int64_t m = 0; m < n; ++m) ptgo_axis_freq(origin, spc, j[m], f, octave, &cell[m], &t[m]);
}

static int dyadic(const ptgo_desc* d) { return d->frequency == 0.0 || d->frequency == 2.0; }

/* ------------------------------------------------------------------------ */
/* Constraint system (Sec. 2.1 Eq. mixedderiv, Sec. 2.2 Eq. polynomial).     */
/* Unknowns: c_a, a in {0..n}^D, index sum_k a_k (n+1)^k.                    */
/* ------------------------------------------------------------------------ */

/* d^d/dx^d of x^a at x (a falling factorial times a power). */
static double dmono(int a, int d, double x)
{
    if (d > a) return 0.0;
    double f = 1.0;
    for (int k = 0; k < d; ++k) f *= (double)(a - k);
    double p = 1.0;
    for (int k = 0; k < a - d; ++k) p *= x;
    return f * p;
}

static int ipow(int b, int e)
{
    int r = 1;
    for (int k = 0; k < e; ++k) r *= b;
    return r;
}

/* Degree per variable and number of unknowns of a method's cell system. */
static int method_degree(int method)
{
    return method == PTGO_C2 ? 5 : 3;
}

static int method_order(int method)
{
    return method == PTGO_C2 ? 2 : 1;
}

/*
 * Build the square constraint matrix of a cell.
 *   Tensor systems (C1: M=1, n=3; C2: M=2, n=5): one row per corner s in
 *   {0,1}^D and per derivative multi-index d with 0 <= d_k <= M, entry
 *   prod_k d^{d_k}/dx^{d_k} x^{a_k} at x = s_k.  The rows with |d| <= M are
 *   the constraints counted by Eq. (nconstraints); the others fix the mixed
 *   derivatives that the paper leaves free (all zero).
 *   Paper gauge (D=2, M=1): the 12 rows with |d| <= 1 plus four rows that
 *   pick c22, c33, c32, c23 (Sec. 3.1).
 * Row metadata rows_meta[r] = (corner s, derivative index d as a base-(M+1)
 * number, or -1 for a gauge row), used to fill right-hand sides.
 * Returns K (rows = columns) or -1.
 */
int ptgo_system(int dims, int method, double* A, int* row_corner, int* row_deriv)
{
    int M = method_order(method), n = method_degree(method);
    int K = ipow(n + 1, dims);
    int ncorner = 1 << dims, nderiv = ipow(M + 1, dims);
    int r = 0;
    if (method == PTGO_PAPER_GAUGE && dims != 2) return -1;
    for (int s = 0; s < ncorner; ++s) {
        for (int di = 0; di < nderiv; ++di) {
            int d[3] = {0, 0, 0}, tot = 0, tmp = di;
            for (int k = 0; k < dims; ++k) {
                d[k] = tmp % (M + 1);
                tmp /= (M + 1);
                tot += d[k];
            }
            if (method == PTGO_PAPER_GAUGE && tot > 1) continue;
            for (int col = 0; col < K; ++col) {
                int a[3] = {0, 0, 0}, tc = col;
                double e = 1.0;
                for (int k = 0; k < dims; ++k) {
                    a[k] = tc % (n + 1);
                    tc /= (n + 1);
                    e *= dmono(a[k], d[k], (double)((s >> k) & 1));
                }
                A[r * K + col] = e;
            }
            row_corner[r] = s;
            row_deriv[r] = di;
            ++r;
        }
    }
    if (method == PTGO_PAPER_GAUGE) {
        /* c22, c33, c32, c23 with c_ij the coefficient of x^i y^j */
        const int gi[4][2] = {{2, 2}, {3, 3}, {3, 2}, {2, 3}};
        for (int g = 0; g < 4; ++g) {
            for (int col = 0; col < K; ++col) A[r * K + col] = 0.0;
            A[r * K + gi[g][0] + gi[g][1] * (n + 1)] = 1.0;
            row_corner[r] = -1;
            row_deriv[r] = -1;
            ++r;
        }
    }
    return r == K ? K : -1;
}

/* Dense LU with partial pivoting, then K solves against unit vectors:
 * Ainv = A^-1.  Returns 0, or -1 if a pivot vanishes. */
int ptgo_invert(int K, const double* A, double* Ainv)
{
    double* LU = (double*)malloc(sizeof(double) * K * K);
    int* piv = (int*)malloc(sizeof(int) * K);
    double* col = (double*)malloc(sizeof(double) * K);
    int rc = 0;
    memcpy(LU, A, sizeof(double) * K * K);
    for (int i = 0; i < K; ++i) piv[i] = i;
    for (int k = 0; k < K && rc == 0; ++k) {
        int p = k;
        double best = fabs(LU[k * K + k]);
        for (int i = k + 1; i < K; ++i)
            if (fabs(LU[i * K + k]) > best) { best = fabs(LU[i * K + k]); p = i; }
        if (best < 1e-300) { rc = -1; break; }
        if (p != k) {
            for (int j = 0; j < K; ++j) {
                double tmp = LU[k * K + j];
                LU[k * K + j] = LU[p * K + j];
                LU[p * K + j] = tmp;
            }
            int tp = piv[k]; piv[k] = piv[p]; piv[p] = tp;
        }
        for (int i = k + 1; i < K; ++i) {
            double l = LU[i * K + k] / LU[k * K + k];
            LU[i * K + k] = l;
            for (int j = k + 1; j < K; ++j) LU[i * K + j] -= l * LU[k * K + j];
        }
    }
    for (int e = 0; e < K && rc == 0; ++e) {
        /* solve A x = unit(e): P A = L U -> L y = P unit(e), U x = y */
        for (int i = 0; i < K; ++i) col[i] = (piv[i] == e) ? 1.0 : 0.0;
        for (int i = 0; i < K; ++i)
            for (int j = 0; j < i; ++j) col[i] -= LU[i * K + j] * col[j];
        for (int i = K - 1; i >= 0; --i) {
            for (int j = i + 1; j < K; ++j) col[i] -= LU[i * K + j] * col[j];
            col[i] /= LU[i * K + i];
        }
        for (int i = 0; i < K; ++i) Ainv[i * K + e] = col[i];
    }
    free(LU);
    free(piv);
    free(col);
    return rc;
}

/* Per-method solved system, built once. */
typedef struct {
    int ready, K;
    double* Ainv;
    int* row_corner;
    int* row_deriv;
} solved_system;

static solved_system g_sys[2][5]; /* [dims-2][method] for methods 1..4 */

static const solved_system* get_system(int dims, int method)
{
    solved_system* S = &g_sys[dims - 2][method];
    if (S->ready) return S;
#ifdef _OPENMP
#pragma omp critical(ptgo_system_build)
#endif
    {
        if (!S->ready) {
            int n = method_degree(method);
            int K = ipow(n + 1, dims);
            double* A = (double*)malloc(sizeof(double) * K * K);
            double* Ainv = (double*)malloc(sizeof(double) * K * K);
            int* rc = (int*)malloc(sizeof(int) * K);
            int* rd = (int*)malloc(sizeof(int) * K);
            if (ptgo_system(dims, method, A, rc, rd) == K && ptgo_invert(K, A, Ainv) == 0) {
                S->K = K;
                S->Ainv = Ainv;
                S->row_corner = rc;
                S->row_deriv = rd;
                __sync_synchronize();
                S->ready = 1;
            }
            free(A);
        }
    }
    return S->ready ? S : NULL;
}

/*
 * Right-hand side of a cell (Sec. 3.1: h_ij, f_ij, g_ij at the corners;
 * Sec. 4: gradients weighted by w).  corner[s*(dims+1) + 0] is the value of
 * corner s, corner[s*(dims+1) + 1 + k] its (unweighted) gradient along k.
 * Value rows take the value, first-derivative rows w times the gradient,
 * every other row zero.
 */
static void cell_rhs(int dims, int method, const solved_system* S, const double* corner, double w,
                     double* rhs)
{
    int M = method_order(method);
    for (int r = 0; r < S->K; ++r) {
        int s = S->row_corner[r], di = S->row_deriv[r];
        double v = 0.0;
        if (s >= 0) {
            int d[3] = {0, 0, 0}, tot = 0, tmp = di, dirk = -1;
            for (int k = 0; k < dims; ++k) {
                d[k] = tmp % (M + 1);
                tmp /= (M + 1);
                tot += d[k];
                if (d[k] == 1) dirk = k;
            }
            if (tot == 0) v = corner[s * (dims + 1)];
            else if (tot == 1) v = w * corner[s * (dims + 1) + 1 + dirk];
        }
        rhs[r] = v;
    }
}

/* Coefficients of one cell: c = A^-1 rhs.  Exported for the pins. */
int ptgo_cell_coeffs(int dims, int method, const double* corner, double w, double* coef)
{
    const solved_system* S = get_system(dims, method);
    if (!S) return -1;
    double rhs[216];
    cell_rhs(dims, method, S, corner, w, rhs);
    for (int i = 0; i < S->K; ++i) {
        double acc = 0.0;
        for (int j = 0; j < S->K; ++j) acc += S->Ainv[i * S->K + j] * rhs[j];
        coef[i] = acc;
    }
    return S->K;
}

/* Eq. (polynomial): h = sum_a c_a prod_k t_k^{a_k}, evaluated term by term. */
static double poly_eval(int dims, int n, const double* coef, const double* t)
{
    int K = ipow(n + 1, dims);
    double h = 0.0;
    for (int col = 0; col < K; ++col) {
        int tc = col;
        double m = 1.0;
        for (int k = 0; k < dims; ++k) {
            int a = tc % (n + 1);
            tc /= (n + 1);
            for (int e = 0; e < a; ++e) m *= t[k];
        }
        h += coef[col] * m;
    }
    return h;
}

/* Smoothstep S3 (Sec. 3.2) and smootherstep S5 (Sec. 5.1). */
static double s3(double x) { return 3.0 * x * x - 2.0 * x * x * x; }
static double s5(double x) { return 6.0 * pow(x, 5) - 15.0 * pow(x, 4) + 10.0 * pow(x, 3); }

/* Corner data of the 2^dims corners of cell `cell` at octave i. */
static void cell_corners(int dims, const uint32_t* cell, uint32_t seed, int octave, double* corner)
{
    for (int s = 0; s < (1 << dims); ++s) {
        uint32_t c[3];
        for (int k = 0; k < dims; ++k) c[k] = cell[k] + (uint32_t)((s >> k) & 1);
        ptgo_corner(dims, c, seed, octave, corner + s * (dims + 1));
    }
}

/* Eq. (zg) with the -xy reading; zero corner gradients. */
static double zero_grad_eval(const double* corner, const double* t)
{
    double h00 = corner[0], h10 = corner[3], h01 = corner[6], h11 = corner[9];
    double x = t[0], y = t[1];
    double dx = h10 - h00, dy = h01 - h00, A = h11 + h00 - h10 - h01;
    return h00 + s3(x) * dx + s3(y) * dy + A * (s3(x) * y + s3(y) * x - x * y);
}

/* Perlin's polynomial (Sec. 3.2): v_ij = f_ij (x - i) + g_ij (y - j), blended
 * along x by S(x), then along y by S(y). */
static double perlin_eval(const double* corner, const double* t, int quintic)
{
    double x = t[0], y = t[1];
    double v[2][2];
    for (int j = 0; j < 2; ++j)
        for (int i = 0; i < 2; ++i) {
            const double* c = corner + (i + 2 * j) * 3;
            v[i][j] = c[1] * (x - i) + c[2] * (y - j);
        }
    double sx = quintic ? s5(x) : s3(x), sy = quintic ? s5(y) : s3(y);
    double h0 = v[0][0] + sx * (v[1][0] - v[0][0]);
    double h1 = v[0][1] + sx * (v[1][1] - v[0][1]);
    return h0 + sy * (h1 - h0);
}

/* Perlin's polynomial in 3D (Sec. 3.2 with a third axis): v_ijk = f (x - i) +
 * g (y - j) + e (z - k) at each of the 8 corners, blended along x by S(x),
 * then along y by S(y), then along z by S(z). */
static double perlin_eval3(const double* corner, const double* t, int quintic)
{
    double v[2][2][2];
    for (int k = 0; k < 2; ++k)
        for (int j = 0; j < 2; ++j)
            for (int i = 0; i < 2; ++i) {
                const double* c = corner + (i + 2 * j + 4 * k) * 4;
                v[i][j][k] = c[1] * (t[0] - i) + c[2] * (t[1] - j) + c[3] * (t[2] - k);
            }
    const double sx = quintic ? s5(t[0]) : s3(t[0]), sy = quintic ? s5(t[1]) : s3(t[1]);
    const double sz = quintic ? s5(t[2]) : s3(t[2]);
    double hz[2];
    for (int k = 0; k < 2; ++k) {
        const double h0 = v[0][0][k] + sx * (v[1][0][k] - v[0][0][k]);
        const double h1 = v[0][1][k] + sx * (v[1][1][k] - v[0][1][k]);
        hz[k] = h0 + sy * (h1 - h0);
    }
    return hz[0] + sz * (hz[1] - hz[0]);
}

/* One octave of a lattice method at (cell, t), t_k in [0, 1] (the cell's own
 * polynomial, also at t = 1 for one-sided difference tests). */
static double lattice_octave(int dims, int method, const uint32_t* cell, const double* t, uint32_t seed,
                             int octave, double w, double* coef_cache, uint32_t* cache_cell, int* cache_ok)
{
    double corner[8 * 4];
    if (method == PTGO_ZERO_GRAD || method == PTGO_PERLIN_S5 || method == PTGO_PERLIN_S3) {
        cell_corners(dims, cell, seed, octave, corner);
        if (method == PTGO_ZERO_GRAD) return zero_grad_eval(corner, t);
        if (dims == 3) return perlin_eval3(corner, t, method == PTGO_PERLIN_S5);
        return perlin_eval(corner, t, method == PTGO_PERLIN_S5);
    }
    int n = method_degree(method);
    int hit = *cache_ok;
    for (int k = 0; k < dims && hit; ++k) hit = (cache_cell[k] == cell[k]);
    if (!hit) {
        cell_corners(dims, cell, seed, octave, corner);
        ptgo_cell_coeffs(dims, method, corner, w, coef_cache);
        for (int k = 0; k < dims; ++k) cache_cell[k] = cell[k];
        *cache_ok = 1;
    }
    return poly_eval(dims, n, coef_cache, t);
}

/* ------------------------------------------------------------------------ */
/* OpenSimplex-style noise: lattice of equilateral triangles with edge       */
/* sqrt(2), obtained by squishing the integer lattice; every vertex within   */
/* distance sqrt(2) of the point adds (2 - r^2)^4 (g . d).  Brute force:     */
/* all vertices of a 7 x 7 block of the stretched lattice around the point.  */
/* ------------------------------------------------------------------------ */
#define OS_STRETCH (-0.21132486540518713)  /* (1/sqrt(3) - 1) / 2 */
#define OS_SQUISH (0.36602540378443865)    /* (sqrt(3) - 1) / 2   */
#define OS_SCALE (0.125)

double ptgo_opensimplex_at(double x, double y, uint32_t seed, int octave)
{
    double s = (x + y) * OS_STRETCH;
    double xs = x + s, ys = y + s;
    int64_t a0 = (int64_t)floor(xs), b0 = (int64_t)floor(ys);
    uint32_t key = octave_key(seed, octave);
    double sum = 0.0;
    for (int da = -3; da <= 3; ++da) {
        for (int db = -3; db <= 3; ++db) {
            int64_t a = a0 + da, b = b0 + db;
            double px = (double)a + (double)(a + b) * OS_SQUISH;
            double py = (double)b + (double)(a + b) * OS_SQUISH;
            double dx = x - px, dy = y - py;
            double r2 = dx * dx + dy * dy;
            if (r2 < 2.0) {
                uint32_t in[3] = {(uint32_t)a, (uint32_t)b, key}, h[3];
                ptgo_pcg3d(in, h);
                double gx = ptgo_unit(h[1]), gy = ptgo_unit(h[2]);
                double k = 2.0 - r2;
                sum += k * k * k * k * (gx * dx + gy * dy);
            }
        }
    }
    return sum * OS_SCALE;
}

/* ------------------------------------------------------------------------ */
/* 3D OpenSimplex-style noise: the same construction one dimension up.       */
/* Squishing Z^3 along its main diagonal by (sqrt(4) - 1)/3 = 1/3 gives a    */
/* lattice whose nearest vertices are sqrt(2) apart (face-centred cubic); a   */
/* point's stretched coordinates are x_k - (x + y + z)/6 (the inverse map).   */
/* Every vertex within distance sqrt(2) adds (2 - r^2)^4 (g . d), g = words   */
/* 1..3 of pcg4d(a, b, c, key).  Brute force over the 7 x 7 x 7 block of the  */
/* stretched lattice around the point (every vertex in range has stretched   */
/* offsets in -1..2 from the point's cell).  Same scale 1/8 as in 2D (the   */
/* raw 3D sum has about the spread of the raw 2D one times 8 as well).       */
/* ------------------------------------------------------------------------ */
/* Sum over the vertices a0 + (da, db, dc) for a point at stretched fraction
 * xi in [0, 1)^3 of cell a0: its displacement from a vertex is u + (sum u)/3
 * per axis, u = xi - (da, db, dc). */
static double os3_sum(const int64_t a0[3], const double xi[3], uint32_t key)
{
    double sum = 0.0;
    for (int da = -3; da <= 3; ++da)
        for (int db = -3; db <= 3; ++db)
            for (int dc = -3; dc <= 3; ++dc) {
                const double u0 = xi[0] - da, u1 = xi[1] - db, u2 = xi[2] - dc;
                const double sq = (u0 + u1 + u2) / 3.0;
                const double d0 = u0 + sq, d1 = u1 + sq, d2 = u2 + sq;
                const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
                if (r2 < 2.0) {
                    uint32_t in[4] = {(uint32_t)(a0[0] + da), (uint32_t)(a0[1] + db), (uint32_t)(a0[2] + dc), key};
                    uint32_t h[4];
                    ptgo_pcg4d(in, h);
                    const double k = 2.0 - r2;
                    sum += k * k * k * k * (ptgo_unit(h[1]) * d0 + ptgo_unit(h[2]) * d1 + ptgo_unit(h[3]) * d2);
                }
            }
    return sum * OS_SCALE;
}

/* At a real lattice position (x, y, z) of octave i. */
double ptgo_opensimplex3_at(double x, double y, double z, uint32_t seed, int octave)
{
    const double sh = -(x + y + z) / 6.0;
    const double s[3] = {x + sh, y + sh, z + sh};
    int64_t a0[3];
    double xi[3];
    for (int k = 0; k < 3; ++k) {
        const double fl = floor(s[k]);
        a0[k] = (int64_t)fl;
        xi[k] = s[k] - fl;
    }
    return os3_sum(a0, xi, octave_key(seed, octave));
}

/* Sample (j_x, j_y, j_z) at octave i of a field with frequency ratio 2:
 * lattice coordinate x_k = I_k + F_k exactly, with the integer
 * I_k = origin_k 2^i + floor(j_k 2^i / spc_k) and the fraction
 * F_k = (j_k 2^i mod spc_k) / spc_k.  Then 6 s_k = (6 I_k - sum I) + (6 F_k -
 * sum F): the stretch needs no rounding at any distance from the origin. */
static double os3_dyadic(const int64_t* origin, const int64_t* spc, const int64_t* j, uint32_t seed, int octave)
{
    int64_t I[3], sumI = 0;
    double F[3], sumF = 0.0;
    for (int k = 0; k < 3; ++k) {
        const int64_t q = j[k] << octave;
        I[k] = origin[k] * ((int64_t)1 << octave) + q / spc[k];
        F[k] = (double)(q % spc[k]) / (double)spc[k];
        sumI += I[k];
        sumF += F[k];
    }
    int64_t a0[3];
    double xi[3];
    for (int k = 0; k < 3; ++k) {
        const double G = 6.0 * F[k] - sumF; /* in (-3, 6) */
        const double fG = floor(G);
        const int64_t T = 6 * I[k] - sumI + (int64_t)fG;
        int64_t a = T / 6;
        if (T - 6 * a < 0) a -= 1; /* floor division */
        a0[k] = a;
        xi[k] = ((double)(T - 6 * a) + (G - fG)) / 6.0;
    }
    return os3_sum(a0, xi, octave_key(seed, octave));
}

/* ------------------------------------------------------------------------ */
/* Fields                                                                    */
/* ------------------------------------------------------------------------ */
static int desc_ok(const ptgo_desc* d)
{
    if (!d || (d->dims != 2 && d->dims != 3) || d->octaves < 1 || d->octaves > 32) return 0;
    if (!(d->frequency == 0.0 || (d->frequency >= 1.0 && d->frequency <= 16.0))) return 0;
    for (int k = 0; k < d->dims; ++k)
        if (d->size[k] <= 0 || d->cells[k] <= 0 || d->size[k] % d->cells[k]) return 0;
    if (d->method == PTGO_C1 || d->method == PTGO_C2 || d->method == PTGO_PERLIN_S5 || d->method == PTGO_PERLIN_S3 ||
        d->method == PTGO_OPENSIMPLEX)
        return 1;
    if (d->dims == 2 && (d->method == PTGO_PAPER_GAUGE || d->method == PTGO_ZERO_GRAD ||
                         d->method == PTGO_PERLIN_S5 || d->method == PTGO_PERLIN_S3 ||
                         d->method == PTGO_OPENSIMPLEX))
        return 1;
    return 0;
}

/*
 * Fractal sum (Sec. 4): H = sum_{i<N} p^i h_i, h_i the octave-i field at the
 * sample.  idx holds n samples, dims integers each (j_x, j_y[, j_z]).
 * Returns 0, or -1 on a bad descriptor.
 */
int ptgo_field_samples(const ptgo_desc* d, const int64_t* idx, int64_t n, double* out, int nthreads)
{
    if (!desc_ok(d)) return -1;
    if (d->method != PTGO_PERLIN_S5 && d->method != PTGO_PERLIN_S3 && d->method != PTGO_OPENSIMPLEX &&
        d->method != PTGO_ZERO_GRAD && !get_system(d->dims, d->method))
        return -1;
    int dims = d->dims;
    int64_t spc[3];
    for (int k = 0; k < dims; ++k) spc[k] = d->size[k] / d->cells[k];
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#else
    (void)nthreads;  /* one thread without OpenMP */
#endif
    {
        double coef[32][216];
        uint32_t ccell[32][3];
        int cok[32];
        for (int i = 0; i < 32; ++i) cok[i] = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int64_t m = 0; m < n; ++m) {
            double H = 0.0, amp = 1.0, weight = 1.0;
            for (int i = 0; i < d->octaves; ++i) {
                uint32_t cell[3];
                double t[3];
                double h;
                for (int k = 0; k < dims; ++k) {
                    if (dyadic(d))
                        ptgo_axis(d->origin[k], spc[k], idx[m * dims + k], i, &cell[k], &t[k]);
                    else
                        ptgo_axis_freq(d->origin[k], spc[k], idx[m * dims + k], d->frequency, i, &cell[k], &t[k]);
                }
                if (d->method == PTGO_OPENSIMPLEX && dims == 3) {
                    if (dyadic(d)) {
                        h = os3_dyadic(d->origin, spc, idx + m * dims, d->seed, i);
                    } else {
                        const double scale = pow(d->frequency, (double)i);
                        double x[3];
                        for (int k = 0; k < 3; ++k)
                            x[k] = ((double)d->origin[k] + (double)idx[m * dims + k] / (double)spc[k]) * scale;
                        h = ptgo_opensimplex3_at(x[0], x[1], x[2], d->seed, i);
                    }
                } else if (d->method == PTGO_OPENSIMPLEX) {
                    /* real position in octave-i lattice units: (origin + j/spc) f^i */
                    double scale = dyadic(d) ? ldexp(1.0, i) : pow(d->frequency, (double)i);
                    double x = ((double)d->origin[0] + (double)idx[m * dims] / (double)spc[0]) * scale;
                    double y = ((double)d->origin[1] + (double)idx[m * dims + 1] / (double)spc[1]) * scale;
                    h = ptgo_opensimplex_at(x, y, d->seed, i);
                } else {
                    h = lattice_octave(dims, d->method, cell, t, d->seed, i, d->grad_weight, coef[i], ccell[i],
                                       &cok[i]);
                }
                if (d->ridged) {
                    /* ridged multifractal: the octave's ridge (1 - |h|)^2,
                     * weighted by the previous octave's weighted ridge times
                     * 2, clamped to [0, 1] */
                    const double ridge = (1.0 - fabs(h)) * (1.0 - fabs(h)) * weight;
                    H += amp * ridge;
                    weight = 2.0 * ridge;
                    if (weight > 1.0) weight = 1.0;
                    if (weight < 0.0) weight = 0.0;
                } else {
                    H += amp * h;
                }
                amp *= d->persistence;
            }
            out[m] = H;
        }
    }
    return 0;
}

/* Whole grid, row-major [z][y][x]. */
int ptgo_field_grid(const ptgo_desc* d, double* out, int nthreads)
{
    if (!desc_ok(d)) return -1;
    int dims = d->dims;
    int64_t total = 1;
    for (int k = 0; k < dims; ++k) total *= d->size[k];
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * total * dims);
    if (!idx) return -1;
    for (int64_t m = 0; m < total; ++m) {
        int64_t r = m;
        for (int k = 0; k < dims; ++k) {
            idx[m * dims + k] = r % d->size[k];
            r /= d->size[k];
        }
    }
    int rc = ptgo_field_samples(d, idx, total, out, nthreads);
    free(idx);
    return rc;
}

/*
 * One octave of a lattice method at explicit (cell, t) points, t_k in [0, 1]
 * (t = 1 evaluates the cell's own polynomial on its far face).  Unscaled by
 * the octave amplitude.  cells: n*dims, t: n*dims.
 */
int ptgo_octave_at(int dims, int method, uint32_t seed, int octave, double w, const uint32_t* cells,
                   const double* t, int64_t n, double* out)
{
    ptgo_desc d;
    memset(&d, 0, sizeof d);
    d.dims = dims;
    d.method = method;
    d.octaves = 1;
    for (int k = 0; k < dims; ++k) d.size[k] = d.cells[k] = 1;
    if (!desc_ok(&d) || method == PTGO_OPENSIMPLEX) return -1;
    if (method != PTGO_PERLIN_S5 && method != PTGO_PERLIN_S3 && method != PTGO_ZERO_GRAD &&
        !get_system(dims, method))
        return -1;
    for (int64_t m = 0; m < n; ++m) {
        double coef[216];
        uint32_t cc[3];
        int ok = 0;
        out[m] = lattice_octave(dims, method, cells + m * dims, t + m * dims, seed, octave, w, coef, cc, &ok);
    }
    return 0;
}

/* OpenSimplex-style noise of one octave at real lattice positions (x, y). */
int ptgo_opensimplex_points(uint32_t seed, int octave, const double* xy, int64_t n, double* out)
{
    for (int64_t m = 0; m < n; ++m) out[m] = ptgo_opensimplex_at(xy[2 * m], xy[2 * m + 1], seed, octave);
    return 0;
}

/* 3D OpenSimplex-style noise of one octave at real lattice positions. */
int ptgo_opensimplex3_points(uint32_t seed, int octave, const double* xyz, int64_t n, double* out)
{
    for (int64_t m = 0; m < n; ++m)
        out[m] = ptgo_opensimplex3_at(xyz[3 * m], xyz[3 * m + 1], xyz[3 * m + 2], seed, octave);
    return 0;
}

/* Batch hash for the bit-exactness tests: n keys of dims+1 words. */
void ptgo_hash_batch(int dims, const uint32_t* keys, int64_t n, uint32_t* out)
{
    for (int64_t m = 0; m < n; ++m) {
        if (dims == 2) ptgo_pcg3d(keys + 3 * m, out + 3 * m);
        else ptgo_pcg4d(keys + 4 * m, out + 4 * m);
    }
}

/* Batch of axis coordinates for the lattice-index tests. */
void ptgo_axis_batch(int64_t origin, int64_t spc, const int64_t* j, int64_t n, int octave, uint32_t* cell, double* t)
{
    for (int64_t m = 0; m < n; ++m) ptgo_axis(origin, spc, j[m], octave, &cell[m], &t[m]);
}

int ptgo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Map statistics of Sec. 5 (the paper's quality measurements).              */
/* ------------------------------------------------------------------------ */

/*
 * Coastline box counting (Sec. 5.3, fractal dimension): squares of side
 * eps = 2^k samples cover the map; a square counts when it holds part of the
 * coastline, i.e. samples below `level` and samples at or above it.  Square
 * (bx, by) covers the samples bx eps .. bx eps + eps (inclusive, clipped to
 * the map) along x, and likewise along y, so neighbouring squares share their
 * edge samples and a crossing between two samples is always inside one
 * square.  There are ceil((W - 1) / eps) x ceil((H - 1) / eps) squares.
 * counts[k] for k = 0 .. levels-1.  h: row-major [H][W].
 */
void ptgo_box_counts(const float* h, int64_t W, int64_t H, float level, int levels, uint64_t* counts)
{
    for (int k = 0; k < levels; ++k) {
        const int64_t eps = (int64_t)1 << k;
        const int64_t nbx = (W - 1 + eps - 1) / eps, nby = (H - 1 + eps - 1) / eps;
        uint64_t n = 0;
        for (int64_t by = 0; by < nby; ++by)
            for (int64_t bx = 0; bx < nbx; ++bx) {
                int below = 0, above = 0;
                const int64_t x1 = bx * eps + eps < W - 1 ? bx * eps + eps : W - 1;
                const int64_t y1 = by * eps + eps < H - 1 ? by * eps + eps : H - 1;
                for (int64_t y = by * eps; y <= y1; ++y)
                    for (int64_t x = bx * eps; x <= x1; ++x) {
                        if (h[y * W + x] < level) below = 1;
                        else above = 1;
                    }
                n += (uint64_t)(below && above);
            }
        counts[k] = n;
    }
}

/*
 * Frequency distribution of heights (what = 0) or of the slope norm
 * (what = 1) over `count` maps of W x H samples ([count][H][W], Sec. 5.1:
 * distributions of height and of the first gradient norm).  The slope at an
 * interior sample is |(central differences in x and y) / 2| in height per
 * sample; border samples have none.  Bins of width (hi - lo) / bins in FP32:
 * b = floor((v - lo) * (bins / (hi - lo))), hist[0] = below lo, hist[1 + b],
 * hist[bins + 1] = at or above hi.  hist has bins + 2 entries, accumulated.
 */
void ptgo_histogram(const float* h, int64_t W, int64_t H, int64_t count, float lo, float hi, int bins, int what,
                    uint64_t* hist)
{
    const float scale = (float)bins / (hi - lo);
    for (int64_t f = 0; f < count; ++f) {
        const float* m = h + f * W * H;
        for (int64_t y = 0; y < H; ++y)
            for (int64_t x = 0; x < W; ++x) {
                float v;
                if (what == 0) {
                    v = m[y * W + x];
                } else {
                    if (x == 0 || y == 0 || x == W - 1 || y == H - 1) continue;
                    const float dx = (m[y * W + x + 1] - m[y * W + x - 1]) * 0.5f;
                    const float dy = (m[(y + 1) * W + x] - m[(y - 1) * W + x]) * 0.5f;
                    const float s2 = dx * dx;
                    const float t2 = dy * dy;
                    v = sqrtf(s2 + t2);
                }
                const float u = (v - lo) * scale;
                const float fb = floorf(u);
                int64_t b;
                if (!(fb >= 0.0f)) b = 0;
                else if (fb >= (float)bins) b = bins + 1;
                else b = (int64_t)fb + 1;
                hist[b] += 1;
            }
    }
}
