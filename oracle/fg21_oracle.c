/*
 * fg21 ORACLE -- test infrastructure only.
 *
 * A plain, slow, FP64 CPU statement of what the region-partitioned global-21cm
 * likelihood computes, written from the paper (arXiv 2603.13196) and sharing no
 * code with the CUDA library.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product path never does.
 *
 * Every routine follows one definition of the paper, cited beside it, with no
 * blocking, fusion or reordering beyond what that definition states.  OpenMP
 * only splits independent outputs (pixels, (f,t) cells or points); every sum
 * runs sequentially in a fixed order, so results do not depend on the thread
 * count.
 *
 * Readings of points the paper leaves open (each stated here in full):
 *  - template map: T230 with nu0 = 230 MHz (Sec. 2.1, eq. of the sky
 *    extrapolation), although eqs. forward_model / chromatic_function print
 *    T408;
 *  - beam: D = 2(p+1) max(0, z.v)^p, zero below the horizon, which makes
 *    (1/4pi) integral D dOmega = 1 as eq. simantenna assumes; the horizon mask
 *    H is that same z.v > 0 test;
 *  - pixel integrals: integral f dOmega = (4 pi / Npix) sum over pixels;
 *  - CDF (eq. weighted_cdf): pixels sorted by (beta asc, index asc), mass of a
 *    pixel = its time- and band-averaged importance; C^-1(c) = beta of the
 *    first sorted pixel whose running mass is >= c;
 *  - regions are (beta_a, beta_b], the lowest one closed below;
 *  - hierarchical splitting uses target masses (k / N_base and their
 *    midpoints) and refines only base regions, which keeps every level exactly
 *    nested (a literal reading of Algorithm 1 can re-split a refined region,
 *    and then level 2^m - 1 is not contained in level 2^m);
 *  - ties: recursive -> largest mass, then lowest beta_a; hierarchical ->
 *    widest, then lowest beta_a;
 *  - N_alpha = 1 (alpha = 1) in the routines without the _ab suffix: the
 *    paper fits spectral-index masks only.  The _ab routines add amplitude
 *    masks M_alpha,i and scale factors alpha_i (eqs. forward_model,
 *    chromatic_function, fast_forward_model); their regions partition a
 *    per-pixel field that the caller supplies (the paper leaves the amplitude
 *    masks' field open; the tests use ln T230), with the same Algorithms and
 *    conventions as the spectral-index masks, and their parameter rows are
 *    [beta_1..beta_Nb, alpha_1..alpha_Na, A21, nu21, sigma21, sigma_n].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_SCHEME_RECURSIVE 0
#define ORC_SCHEME_HIERARCHICAL 1
#define ORC_SCHEME_LINEAR 2
#define ORC_SCHEME_PERCENTILE 3

#define ORC_WEIGHT_BEAM 0
#define ORC_WEIGHT_SKY 1
#define ORC_WEIGHT_HORIZON 2
#define ORC_WEIGHT_UNIFORM 3

/* ---------------------------------------------------------------- beam */

/* Directivity of the synthetic beam at pixel direction v for zenith z and
 * exponent p: 2(p+1) cos(zenith angle)^p above the horizon, 0 below
 * (eq. simantenna's D, with the static horizon H folded in). */
static double orc_beam(const double *v, const double *z, double p)
{
    double c = v[0] * z[0] + v[1] * z[1] + v[2] * z[2];
    if (c <= 0.0) return 0.0;
    return 2.0 * (p + 1.0) * pow(c, p);
}

/* Sky temperature of one pixel at frequency nu (Sec. 2.1, eq. skyapproximation):
 * (T230 - T_CMB) (nu/nu0)^-beta + T_CMB. */
static double orc_tsky(double t230, double beta, double nu, double nu0, double t_cmb)
{
    return (t230 - t_cmb) * pow(nu / nu0, -beta) + t_cmb;
}

/* Gaussian 21-cm trough (Sec. 2.1, eq. t21model). */
double orc_t21(double nu, double a21, double nu21, double s21)
{
    double d = nu - nu21;
    return a21 * exp(-(d * d) / (2.0 * s21 * s21));
}

/* ------------------------------------------------- importance weighting */

/* Per-pixel importance averaged over band and LST (Sec. 4.2):
 *   W(pix,f,t) = num(pix,f,t) / sum_q num(q,f,t)
 *   beam    : num = T_sky D H            (eq. w_beam_dynamic)
 *   sky     : num = T_sky H
 *   horizon : num = H
 *   uniform : num = 1                    (observation independent)
 * and w[pix] = (1/(F T)) sum_f sum_t W(pix,f,t), f outer, t inner, ascending.
 * The (4pi/Npix) of the discrete integrals cancels in the ratio.
 * Scratch den[F*T] is allocated here. */
int orc_weights(int64_t npix, const double *dirs, const double *t230, const double *beta,
                int F, const double *nu, double nu0, int T, const double *zenith,
                const double *beam_p, double t_cmb, int weighting, double *w_out)
{
    double *den = (double *)calloc((size_t)F * T, sizeof(double));
    if (!den) return -2;
#pragma omp parallel for schedule(dynamic)
    for (int ft = 0; ft < F * T; ++ft) {
        int f = ft / T, t = ft % T;
        double s = 0.0;
        for (int64_t q = 0; q < npix; ++q) {
            const double *v = dirs + 3 * q;
            const double *z = zenith + 3 * t;
            double num;
            double c = v[0] * z[0] + v[1] * z[1] + v[2] * z[2];
            if (weighting == ORC_WEIGHT_BEAM)
                num = orc_tsky(t230[q], beta[q], nu[f], nu0, t_cmb) * orc_beam(v, z, beam_p[f]);
            else if (weighting == ORC_WEIGHT_SKY)
                num = c > 0.0 ? orc_tsky(t230[q], beta[q], nu[f], nu0, t_cmb) : 0.0;
            else if (weighting == ORC_WEIGHT_HORIZON)
                num = c > 0.0 ? 1.0 : 0.0;
            else
                num = 1.0;
            s += num;
        }
        den[ft] = s;
    }
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < npix; ++q) {
        const double *v = dirs + 3 * q;
        double acc = 0.0;
        for (int f = 0; f < F; ++f) {
            for (int t = 0; t < T; ++t) {
                const double *z = zenith + 3 * t;
                double c = v[0] * z[0] + v[1] * z[1] + v[2] * z[2];
                double num;
                if (weighting == ORC_WEIGHT_BEAM)
                    num = orc_tsky(t230[q], beta[q], nu[f], nu0, t_cmb) * orc_beam(v, z, beam_p[f]);
                else if (weighting == ORC_WEIGHT_SKY)
                    num = c > 0.0 ? orc_tsky(t230[q], beta[q], nu[f], nu0, t_cmb) : 0.0;
                else if (weighting == ORC_WEIGHT_HORIZON)
                    num = c > 0.0 ? 1.0 : 0.0;
                else
                    num = 1.0;
                double d = den[f * T + t];
                acc += d > 0.0 ? num / d : 0.0;
            }
        }
        w_out[q] = acc / ((double)F * (double)T);
    }
    free(den);
    return 0;
}

/* ------------------------------------------------------------ partition */

static const double *g_sort_beta;
static int cmp_beta_idx(const void *a, const void *b)
{
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    double bi = g_sort_beta[i], bj = g_sort_beta[j];
    if (bi < bj) return -1;
    if (bi > bj) return 1;
    return (i > j) - (i < j);
}

/* Pixel order of the discrete CDF: beta ascending, then index ascending. */
void orc_sorted_order(int64_t npix, const double *beta, int64_t *order)
{
    for (int64_t k = 0; k < npix; ++k) order[k] = k;
    g_sort_beta = beta;
    qsort(order, (size_t)npix, sizeof(int64_t), cmp_beta_idx);
}

/* Margin bookkeeping: the smallest relative gap of any comparison that decided
 * the partition (near-ties would let rounding differences flip a label). */
static void margin_update(double *m, double a, double b)
{
    double scale = fabs(a) > fabs(b) ? fabs(a) : fabs(b);
    if (scale == 0.0) return;          /* exact tie of zeros: decided by the tie rule */
    double r = fabs(a - b) / scale;
    if (r < *m) *m = r;
}

/* C^-1(c): beta of the first sorted pixel whose running mass reaches c. */
static double orc_cinv(int64_t npix, const int64_t *order, const double *beta,
                       const double *cum, double c, double *margin)
{
    for (int64_t k = 0; k < npix; ++k) {
        if (cum[k] >= c) {
            margin_update(margin, cum[k], c);
            if (k > 0) margin_update(margin, cum[k - 1], c);
            return beta[order[k]];
        }
    }
    return beta[order[npix - 1]];
}

/* Mass of region (a, b] (closed below if lowest): sum of w over its pixels,
 * summed in sorted order (eq. weighted_cdf: m_r = integral over r of dC). */
static double orc_region_mass(int64_t npix, const int64_t *order, const double *beta,
                              const double *w, double a, double b, int lowest)
{
    double m = 0.0;
    for (int64_t k = 0; k < npix; ++k) {
        double x = beta[order[k]];
        int in = (x <= b) && (lowest ? x >= a : x > a);
        if (in) m += w[order[k]];
    }
    return m;
}

/* `lowest` marks the region closed below (recursive scheme) or an unsplit
 * base region (hierarchical scheme). */
typedef struct { double a, b, ca, cb; int lowest; } orc_region;

static int cmp_region(const void *x, const void *y)
{
    const orc_region *r = (const orc_region *)x, *s = (const orc_region *)y;
    if (r->a < s->a) return -1;
    if (r->a > s->a) return 1;
    if (r->b < s->b) return -1;
    if (r->b > s->b) return 1;
    return 0;
}

/* Partition the beta axis into N regions and label every pixel.
 *  recursive    : Algorithm 2 (Sec. 4.3.2) -- start from [beta_min, beta_max],
 *                 repeatedly bisect the region of largest mass at its beta
 *                 midpoint;
 *  hierarchical : Algorithm 1 (Sec. 4.3.1) -- N_base = 2^floor(log2 N) equal-mass
 *                 regions, then bisect the widest not-yet-bisected base region
 *                 at its importance midpoint C^-1((c_a + c_b)/2);
 *  linear       : N equal-width beta intervals (Sec. 4.1 (i));
 *  percentile   : N intervals of equal pixel count (Sec. 4.1 (ii)).
 * edges[N+1] ascending; labels[pix] = number of interior edges below beta.
 * *margin = smallest relative gap of a deciding comparison (1 if none). */
int orc_partition(int64_t npix, const double *beta, const double *w, int N, int scheme,
                  double *edges, int32_t *labels, double *margin)
{
    if (N < 1 || npix < 1) return -1;
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)npix);
    double *cum = (double *)malloc(sizeof(double) * (size_t)npix);
    orc_region *R = (orc_region *)malloc(sizeof(orc_region) * (size_t)(N + 1));
    if (!order || !cum || !R) { free(order); free(cum); free(R); return -2; }
    orc_sorted_order(npix, beta, order);
    double run = 0.0;
    for (int64_t k = 0; k < npix; ++k) { run += w[order[k]]; cum[k] = run; }
    double bmin = beta[order[0]], bmax = beta[order[npix - 1]];
    *margin = 1.0;
    int nR = 0;

    if (scheme == ORC_SCHEME_RECURSIVE) {
        R[0].a = bmin; R[0].b = bmax; R[0].ca = 0.0; R[0].cb = 1.0; R[0].lowest = 1; nR = 1;
        while (nR < N) {
            double *m = (double *)malloc(sizeof(double) * (size_t)nR);
            for (int r = 0; r < nR; ++r)
                m[r] = orc_region_mass(npix, order, beta, w, R[r].a, R[r].b, R[r].lowest);
            int best = 0;
            for (int r = 1; r < nR; ++r)
                if (m[r] > m[best] || (m[r] == m[best] && R[r].a < R[best].a)) best = r;
            for (int r = 0; r < nR; ++r)
                if (r != best) margin_update(margin, m[best], m[r]);
            free(m);
            double a = R[best].a, b = R[best].b, mid = 0.5 * (a + b);
            R[best].b = mid;
            R[nR].a = mid; R[nR].b = b; R[nR].ca = 0.0; R[nR].cb = 0.0; R[nR].lowest = 0;
            ++nR;
        }
    } else if (scheme == ORC_SCHEME_HIERARCHICAL) {
        int nb = 1;
        while (nb * 2 <= N) nb *= 2;
        double prev_b = bmin, prev_c = 0.0;
        for (int j = 1; j <= nb; ++j) {
            double c = (double)j / (double)nb;
            double e = (j == nb) ? bmax : orc_cinv(npix, order, beta, cum, c, margin);
            R[nR].a = prev_b; R[nR].b = e; R[nR].ca = prev_c; R[nR].cb = c; ++nR;
            prev_b = e; prev_c = c;
        }
        /* refinement: bisect the widest base region not yet bisected (a
         * region made by an earlier refinement is never split again, which is
         * what keeps level 2^m - 1 inside the 2^m base partition) */
        for (int r = 0; r < nR; ++r) R[r].lowest = 1;          /* flag: unsplit base region */
        while (nR < N) {
            int best = -1;
            for (int r = 0; r < nR; ++r) {
                if (!R[r].lowest) continue;
                if (best < 0) { best = r; continue; }
                double wr = R[r].b - R[r].a, wb = R[best].b - R[best].a;
                if (wr > wb || (wr == wb && R[r].a < R[best].a)) best = r;
            }
            for (int r = 0; r < nR; ++r)
                if (r != best && R[r].lowest)
                    margin_update(margin, R[best].b - R[best].a, R[r].b - R[r].a);
            double cm = 0.5 * (R[best].ca + R[best].cb);
            double bm = orc_cinv(npix, order, beta, cum, cm, margin);
            double b = R[best].b, cb = R[best].cb;
            R[best].b = bm; R[best].cb = cm; R[best].lowest = 0;
            R[nR].a = bm; R[nR].b = b; R[nR].ca = cm; R[nR].cb = cb; R[nR].lowest = 0; ++nR;
        }
    } else if (scheme == ORC_SCHEME_LINEAR) {
        for (int j = 0; j < N; ++j) {
            R[j].a = (j == 0) ? bmin : bmin + (bmax - bmin) * (double)j / (double)N;
            R[j].b = (j == N - 1) ? bmax : bmin + (bmax - bmin) * (double)(j + 1) / (double)N;
        }
        nR = N;
    } else if (scheme == ORC_SCHEME_PERCENTILE) {
        double prev = bmin;
        for (int j = 1; j <= N; ++j) {
            /* first sorted position k with (k+1)/Npix >= j/N */
            int64_t k = ((int64_t)j * npix + N - 1) / N - 1;
            double e = (j == N) ? bmax : beta[order[k]];
            R[j - 1].a = prev; R[j - 1].b = e; prev = e;
        }
        nR = N;
    } else {
        free(order); free(cum); free(R);
        return -1;
    }

    qsort(R, (size_t)nR, sizeof(orc_region), cmp_region);
    edges[0] = bmin;
    for (int j = 0; j < N; ++j) edges[j + 1] = R[j].b;
    for (int64_t q = 0; q < npix; ++q) {
        int lab = 0;
        for (int j = 1; j < N; ++j)
            if (beta[q] > edges[j]) lab = j;
        labels[q] = lab;
    }
    free(order); free(cum); free(R);
    return 0;
}

/* ----------------------------------------------------------- precompute */

/* Chromatic response functions (Sec. 2.2, eq. chromatic_function, N_alpha = 1)
 * and the beam normalisation that multiplies T_CMB in eq. fast_forward_model:
 *   A[i,f,t] = (1/Npix) sum_{pix in region i} (T230 - T_CMB) D(pix,f,t)
 *   B[f,t]   = (1/Npix) sum_pix D(pix,f,t)
 * Sums run over pixels in index order, one (f,t) cell at a time. */
int orc_precompute(int64_t npix, const double *dirs, const double *t230, const int32_t *labels,
                   int N, int F, int T, const double *zenith, const double *beam_p, double t_cmb,
                   double *A, double *B)
{
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * (size_t)N);
#pragma omp for schedule(dynamic)
        for (int ft = 0; ft < F * T; ++ft) {
            int f = ft / T, t = ft % T;
            for (int i = 0; i < N; ++i) acc[i] = 0.0;
            double b = 0.0;
            for (int64_t q = 0; q < npix; ++q) {
                double d = orc_beam(dirs + 3 * q, zenith + 3 * t, beam_p[f]);
                acc[labels[q]] += (t230[q] - t_cmb) * d;
                b += d;
            }
            for (int i = 0; i < N; ++i) A[((size_t)i * F + f) * T + t] = acc[i] / (double)npix;
            B[(size_t)f * T + t] = b / (double)npix;
        }
        free(acc);
    }
    return 0;
}

/* --------------------------------------------------------- forward model */

/* Fast forward model (Sec. 2.2, eq. fast_forward_model, with the discrete B)
 * plus the 21-cm trough (eq. likelihood's M = T_FG + T21):
 *   M[p,f,t] = sum_i A[i,f,t] (nu_f/nu0)^-beta_{p,i} + T_CMB B[f,t] + T21(nu_f)
 * params rows: [beta_1..beta_N, A21, nu21, sigma21, sigma_n]. */
void orc_fast_model(int N, int F, int T, const double *A, const double *B, const double *nu,
                    double nu0, double t_cmb, const double *params, int64_t P, double *M)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < P; ++p) {
        const double *th = params + (size_t)p * (N + 4);
        for (int f = 0; f < F; ++f) {
            double s21 = orc_t21(nu[f], th[N], th[N + 1], th[N + 2]);
            for (int t = 0; t < T; ++t) {
                double fg = 0.0;
                for (int i = 0; i < N; ++i)
                    fg += A[((size_t)i * F + f) * T + t] * pow(nu[f] / nu0, -th[i]);
                M[((size_t)p * F + f) * T + t] = fg + t_cmb * B[(size_t)f * T + t] + s21;
            }
        }
    }
}

/* Per-pixel forward model (Sec. 2.2, eq. forward_model) convolved with the beam
 * (eq. simantenna's integral), without the precomputed A:
 *   M[p,f,t] = (1/Npix) sum_pix D [(T230 - T_CMB)(nu/nu0)^-beta_{p,label(pix)} + T_CMB]
 *              + T21(nu_f).
 * The second route to the same numbers, for pinning orc_precompute. */
void orc_pixel_model(int64_t npix, const double *dirs, const double *t230, const int32_t *labels,
                     int N, int F, const double *nu, double nu0, int T, const double *zenith,
                     const double *beam_p, double t_cmb, const double *params, int64_t P, double *M)
{
#pragma omp parallel for schedule(dynamic)
    for (int64_t pft = 0; pft < P * F * T; ++pft) {
        int64_t p = pft / ((int64_t)F * T);
        int f = (int)((pft / T) % F), t = (int)(pft % T);
        const double *th = params + (size_t)p * (N + 4);
        double s = 0.0;
        for (int64_t q = 0; q < npix; ++q) {
            double d = orc_beam(dirs + 3 * q, zenith + 3 * t, beam_p[f]);
            double tm = (t230[q] - t_cmb) * pow(nu[f] / nu0, -th[labels[q]]) + t_cmb;
            s += d * tm;
        }
        M[pft] = s / (double)npix + orc_t21(nu[f], th[N], th[N + 1], th[N + 2]);
    }
}

/* Simulated antenna temperature (Sec. 2.1, eq. simantenna) with the per-pixel
 * spectral index of the sky:
 *   data[f,t] = (1/Npix) sum_pix D T_sky(pix,f) + T21(nu_f) + sigma_noise * noise[f,t]. */
void orc_simulate_data(int64_t npix, const double *dirs, const double *t230, const double *beta,
                       int F, const double *nu, double nu0, int T, const double *zenith,
                       const double *beam_p, double t_cmb, const double *t21p,
                       double sigma_noise, const double *noise, double *data)
{
#pragma omp parallel for schedule(dynamic)
    for (int ft = 0; ft < F * T; ++ft) {
        int f = ft / T, t = ft % T;
        double s = 0.0;
        for (int64_t q = 0; q < npix; ++q)
            s += orc_beam(dirs + 3 * q, zenith + 3 * t, beam_p[f]) *
                 orc_tsky(t230[q], beta[q], nu[f], nu0, t_cmb);
        double v = s / (double)npix + orc_t21(nu[f], t21p[0], t21p[1], t21p[2]);
        if (noise) v += sigma_noise * noise[ft];
        data[ft] = v;
    }
}

/* ------------------------------------------------------------ likelihood */

/* Gaussian log-likelihood with free sigma_n (Sec. 2.3.1, eq. likelihood):
 *   lnL = -1/2 sum_{f,t} [ ln(2 pi sigma_n^2) + (D - M)^2 / sigma_n^2 ].
 * M is the fast forward model of orc_fast_model, evaluated point by point. */
void orc_loglike(int N, int F, int T, const double *A, const double *B, const double *data,
                 const double *nu, double nu0, double t_cmb, const double *params, int64_t P,
                 double *logL)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < P; ++p) {
        const double *th = params + (size_t)p * (N + 4);
        double sig = th[N + 3];
        double sum = 0.0;
        for (int f = 0; f < F; ++f) {
            double s21 = orc_t21(nu[f], th[N], th[N + 1], th[N + 2]);
            for (int t = 0; t < T; ++t) {
                double fg = 0.0;
                for (int i = 0; i < N; ++i)
                    fg += A[((size_t)i * F + f) * T + t] * pow(nu[f] / nu0, -th[i]);
                double m = fg + t_cmb * B[(size_t)f * T + t] + s21;
                double r = data[(size_t)f * T + t] - m;
                sum += log(2.0 * 3.14159265358979323846 * sig * sig) + r * r / (sig * sig);
            }
        }
        logL[p] = -0.5 * sum;
    }
}

/* Chi-square part only, sum (D - M)^2, for tolerance bookkeeping. */
void orc_chi2(int N, int F, int T, const double *A, const double *B, const double *data,
              const double *nu, double nu0, double t_cmb, const double *params, int64_t P,
              double *chi2)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < P; ++p) {
        const double *th = params + (size_t)p * (N + 4);
        double sum = 0.0;
        for (int f = 0; f < F; ++f) {
            double s21 = orc_t21(nu[f], th[N], th[N + 1], th[N + 2]);
            for (int t = 0; t < T; ++t) {
                double fg = 0.0;
                for (int i = 0; i < N; ++i)
                    fg += A[((size_t)i * F + f) * T + t] * pow(nu[f] / nu0, -th[i]);
                double r = data[(size_t)f * T + t] - (fg + t_cmb * B[(size_t)f * T + t] + s21);
                sum += r * r;
            }
        }
        chi2[p] = sum;
    }
}

/* ------------------------------------------------------- amplitude masks */

/* Chromatic response functions with both sets of masks (Sec. 2.2, eq.
 * chromatic_function, dOmega = 4 pi / Npix):
 *   K[i,j,f,t] = (1/Npix) sum_pix M_alpha,i(pix) M_beta,j(pix) (T230 - T_CMB) D(pix,f,t)
 * with M_alpha,i(pix) = [lab_a(pix) == i] and M_beta,j(pix) = [lab_b(pix) == j].
 * K is [Na][Nb][F][T].  B[f,t] = (1/Npix) sum_pix D as in orc_precompute.
 * Each (i, j, f, t) sums over all pixels in index order. */
int orc_precompute_ab(int64_t npix, const double *dirs, const double *t230, const int32_t *lab_a, int Na,
                      const int32_t *lab_b, int Nb, int F, int T, const double *zenith,
                      const double *beam_p, double t_cmb, double *K, double *B)
{
#pragma omp parallel for schedule(dynamic)
    for (int ft = 0; ft < F * T; ++ft) {
        int f = ft / T, t = ft % T;
        for (int i = 0; i < Na; ++i) {
            for (int j = 0; j < Nb; ++j) {
                double s = 0.0;
                for (int64_t q = 0; q < npix; ++q) {
                    double ma = lab_a[q] == i ? 1.0 : 0.0;
                    double mb = lab_b[q] == j ? 1.0 : 0.0;
                    s += ma * mb * (t230[q] - t_cmb) * orc_beam(dirs + 3 * q, zenith + 3 * t, beam_p[f]);
                }
                K[(((size_t)i * Nb + j) * F + f) * T + t] = s / (double)npix;
            }
        }
        double b = 0.0;
        for (int64_t q = 0; q < npix; ++q) b += orc_beam(dirs + 3 * q, zenith + 3 * t, beam_p[f]);
        B[(size_t)f * T + t] = b / (double)npix;
    }
    return 0;
}

/* Foreground of eq. fast_forward_model for one parameter row at (f, t):
 *   sum_i sum_j alpha_i K[i,j,f,t] (nu_f/nu0)^-beta_j. */
static double orc_fg_ab(int Na, int Nb, int F, int T, const double *K, const double *nu, double nu0,
                        const double *th, int f, int t)
{
    double fg = 0.0;
    for (int i = 0; i < Na; ++i)
        for (int j = 0; j < Nb; ++j)
            fg += th[Nb + i] * K[(((size_t)i * Nb + j) * F + f) * T + t] * pow(nu[f] / nu0, -th[j]);
    return fg;
}

/* Fast forward model with amplitude masks (eq. fast_forward_model with the
 * discrete B) plus the trough:
 *   M[p,f,t] = sum_i sum_j alpha_i K[i,j,f,t] (nu_f/nu0)^-beta_j + T_CMB B[f,t] + T21(nu_f).
 * params rows: [beta_1..beta_Nb, alpha_1..alpha_Na, A21, nu21, sigma21, sigma_n]. */
void orc_fast_model_ab(int Na, int Nb, int F, int T, const double *K, const double *B, const double *nu,
                       double nu0, double t_cmb, const double *params, int64_t P, double *M)
{
    const int NP = Nb + Na;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < P; ++p) {
        const double *th = params + (size_t)p * (NP + 4);
        for (int f = 0; f < F; ++f) {
            double s21 = orc_t21(nu[f], th[NP], th[NP + 1], th[NP + 2]);
            for (int t = 0; t < T; ++t)
                M[((size_t)p * F + f) * T + t] =
                    orc_fg_ab(Na, Nb, F, T, K, nu, nu0, th, f, t) + t_cmb * B[(size_t)f * T + t] + s21;
        }
    }
}

/* Per-pixel forward model with amplitude masks (eq. forward_model) integrated
 * against the beam (eq. simantenna's integral), without K:
 *   M[p,f,t] = (1/Npix) sum_pix D [alpha_{lab_a(pix)} (T230 - T_CMB)(nu/nu0)^-beta_{lab_b(pix)}
 *              + T_CMB] + T21(nu_f). */
void orc_pixel_model_ab(int64_t npix, const double *dirs, const double *t230, const int32_t *lab_a, int Na,
                        const int32_t *lab_b, int Nb, int F, const double *nu, double nu0, int T,
                        const double *zenith, const double *beam_p, double t_cmb, const double *params,
                        int64_t P, double *M)
{
    const int NP = Nb + Na;
#pragma omp parallel for schedule(dynamic)
    for (int64_t pft = 0; pft < P * F * T; ++pft) {
        int64_t p = pft / ((int64_t)F * T);
        int f = (int)((pft / T) % F), t = (int)(pft % T);
        const double *th = params + (size_t)p * (NP + 4);
        double s = 0.0;
        for (int64_t q = 0; q < npix; ++q) {
            double d = orc_beam(dirs + 3 * q, zenith + 3 * t, beam_p[f]);
            double tm = th[Nb + lab_a[q]] * (t230[q] - t_cmb) * pow(nu[f] / nu0, -th[lab_b[q]]) + t_cmb;
            s += d * tm;
        }
        M[pft] = s / (double)npix + orc_t21(nu[f], th[NP], th[NP + 1], th[NP + 2]);
    }
}

/* Gaussian log-likelihood (Sec. 2.3.1, eq. likelihood) over the model of
 * orc_fast_model_ab:
 *   lnL = -1/2 sum_{f,t} [ ln(2 pi sigma_n^2) + (D - M)^2 / sigma_n^2 ]. */
void orc_loglike_ab(int Na, int Nb, int F, int T, const double *K, const double *B, const double *data,
                    const double *nu, double nu0, double t_cmb, const double *params, int64_t P, double *logL)
{
    const int NP = Nb + Na;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < P; ++p) {
        const double *th = params + (size_t)p * (NP + 4);
        double sig = th[NP + 3];
        double sum = 0.0;
        for (int f = 0; f < F; ++f) {
            double s21 = orc_t21(nu[f], th[NP], th[NP + 1], th[NP + 2]);
            for (int t = 0; t < T; ++t) {
                double m = orc_fg_ab(Na, Nb, F, T, K, nu, nu0, th, f, t) + t_cmb * B[(size_t)f * T + t] + s21;
                double r = data[(size_t)f * T + t] - m;
                sum += log(2.0 * 3.14159265358979323846 * sig * sig) + r * r / (sig * sig);
            }
        }
        logL[p] = -0.5 * sum;
    }
}

/* Chi-square part only, sum (D - M)^2 over the model of orc_fast_model_ab. */
void orc_chi2_ab(int Na, int Nb, int F, int T, const double *K, const double *B, const double *data,
                 const double *nu, double nu0, double t_cmb, const double *params, int64_t P, double *chi2)
{
    const int NP = Nb + Na;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < P; ++p) {
        const double *th = params + (size_t)p * (NP + 4);
        double sum = 0.0;
        for (int f = 0; f < F; ++f) {
            double s21 = orc_t21(nu[f], th[NP], th[NP + 1], th[NP + 2]);
            for (int t = 0; t < T; ++t) {
                double r = data[(size_t)f * T + t] -
                           (orc_fg_ab(Na, Nb, F, T, K, nu, nu0, th, f, t) + t_cmb * B[(size_t)f * T + t] + s21);
                sum += r * r;
            }
        }
        chi2[p] = sum;
    }
}

/* ------------------------------------------ noise-only likelihood (q_i) */

/* Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11, "Parallel random
 * numbers: as easy as 1, 2, 3"): ten rounds of two 32x32 -> 64-bit products
 * with multipliers 0xD2511F53 and 0xCD9E8D57, the Feistel-like mixing
 *   (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
 * and the key bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85) between
 * rounds.  The counter-based generator both sides implement from this
 * definition; the noise realisations of the accuracy criterion are drawn
 * from it. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Standard-normal draws z[cell] of noise realisation k: cells are taken in
 * pairs (2j, 2j+1); pair j of realisation k uses Philox4x32-10 with counter
 * (j, k mod 2^32, k / 2^32, 0) and key (seed mod 2^32, seed / 2^32), its
 * first two outputs as uniforms u = (x + 1) / 2^32 in (0, 1], and the
 * Box-Muller transform z_2j = sqrt(-2 ln u1) cos(2 pi u2),
 * z_2j+1 = sqrt(-2 ln u1) sin(2 pi u2) (the second is dropped for an odd last
 * cell).  z [n_cells]. */
static void orc_noise_draws_one(int64_t n_cells, int64_t k, uint64_t seed, double *z)
{
    const double two_pi = 6.28318530717958647692;
    for (int64_t j = 0; 2 * j < n_cells; ++j) {
        uint32_t ctr[4] = {(uint32_t)j, (uint32_t)k, (uint32_t)((uint64_t)k >> 32), 0u};
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        uint32_t x[4];
        orc_philox4x32_10(ctr, key, x);
        double u1 = ((double)x[0] + 1.0) / 4294967296.0;
        double u2 = ((double)x[1] + 1.0) / 4294967296.0;
        double r = sqrt(-2.0 * log(u1));
        z[2 * j] = r * cos(two_pi * u2);
        if (2 * j + 1 < n_cells) z[2 * j + 1] = r * sin(two_pi * u2);
    }
}

/* The draws of realisations 0..K-1: out [K][n_cells]. */
void orc_noise_draws(int64_t n_cells, int64_t K, uint64_t seed, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < K; ++k) orc_noise_draws_one(n_cells, k, seed, out + k * n_cells);
}

/* The likelihood distribution of the accuracy criterion (Sec. 5.2.2: data
 * described perfectly by the model up to noise realisations): for each
 * realisation k the residual D - M is the noise itself, sigma_noise z[k], so
 * eq. likelihood gives
 *   L_noise[k] = -1/2 sum_cells [ ln(2 pi sigma_n^2) + (sigma_noise z[k,cell])^2 / sigma_n^2 ],
 * summed over cells in order. */
void orc_noise_loglike(int64_t n_cells, double sigma_noise, double sigma_n, int64_t K, uint64_t seed,
                       double *L_noise)
{
    const double lnorm = log(2.0 * 3.14159265358979323846 * sigma_n * sigma_n);
#pragma omp parallel
    {
        double *z = (double *)malloc(sizeof(double) * (size_t)n_cells);
#pragma omp for schedule(dynamic, 16)
        for (int64_t k = 0; k < K; ++k) {
            orc_noise_draws_one(n_cells, k, seed, z);
            double sum = 0.0;
            for (int64_t c = 0; c < n_cells; ++c) {
                double res = sigma_noise * z[c];
                sum += lnorm + res * res / (sigma_n * sigma_n);
            }
            L_noise[k] = -0.5 * sum;
        }
        free(z);
    }
}

/* q = P(L_noise <= L_bar) of Sec. 5.2.2: the fraction of the K realisations
 * whose likelihood does not exceed L_bar (the lower-tail probability of the
 * fitted likelihood under the ideal noise distribution), for each of n_bar
 * values L_bar. */
void orc_noise_q(const double *L_noise, int64_t K, const double *L_bar, int64_t n_bar, double *q)
{
    for (int64_t i = 0; i < n_bar; ++i) {
        int64_t c = 0;
        for (int64_t k = 0; k < K; ++k) c += L_noise[k] <= L_bar[i];
        q[i] = (double)c / (double)K;
    }
}
