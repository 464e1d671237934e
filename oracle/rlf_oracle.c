/*
 * FP64 CPU oracle for the RadioLensfit hot path (Rivi & Miller, arXiv 2203.14071).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  The CUDA library shares no code,
 * header, table or constant generator with it.
 *
 * Every routine is the plain definition of one step of the method, written in
 * double precision with straightforward loops:
 *   rlfo_model_vis      Eq. 1 with the shear matrix of Eq. 2 (Sec. 2.2)
 *   rlfo_alpha_med      Eq. 4 scale-flux relation (Sec. 2.2)
 *   rlfo_sky_model      sum of Eq. 1 over the catalogue (Sec. 2.2)
 *   rlfo_simulate_vis   the same sum, arranged for speed, to make test data
 *   rlfo_extract_facet  residual isolation, phase shift and facet averaging
 *                       (Sec. 2.3), facet size K * alpha (Sec. 2.3, Sec. 4.1)
 *   rlfo_fit_facet      chi^2 likelihood, analytic flux marginal, numeric
 *                       scalelength marginal, 5% threshold moments and the
 *                       bad-fit cut (Sec. 2.4, Sec. 4.1); with n_pos > 1 the
 *                       position marginal over a grid of offsets (Sec. 2.4)
 *   rlfo_fit_facet_adaptive  the estimate on halved lattices around the kept
 *                       samples (adaptive sampling, Sec. 2.4)
 *   rlfo_pipeline       the whole chain with the sky-model update in chunks
 *                       (Sec. 2.2, Sec. 3.1), and the refit of bad fits (Sec. 2.4)
 * Readings where the paper is silent are stated beside the code that takes them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define RLFO_C 299792458.0
#define RLFO_PI 3.14159265358979323846
#define RLFO_ARCSEC (RLFO_PI / 648000.0)

/* per-source estimate record written by rlfo_fit_facet */
enum {
    RLFO_E1 = 0, RLFO_E2, RLFO_SIG1, RLFO_SIG2, RLFO_ALPHA, RLFO_FLUX, RLFO_FLAG,
    RLFO_E1_SMOOTH, RLFO_E2_SMOOTH, RLFO_LOGL_MAX, RLFO_THRESH_MARGIN, RLFO_MAP_INDEX,
    RLFO_NC, RLFO_LEVELS, RLFO_STEP, RLFO_NKEPT, RLFO_REFIT, RLFO_NEST
};

typedef struct {
    double add, esp, psf_nat, beta, nu_ref_hz, sigma_jy;
    double e_max, r_min_arcsec, r_max_arcsec, r_std;
    double thresh_frac, var_sigma_min, var_det_min;
    int32_t facet_n, n_e, n_alpha, flux_prior; /* flux_prior 0: S in [0, inf); 1: real line */
    int32_t chunk, update_mode;                /* update_mode 0: good fits only; 1: all */
    int32_t profile, pad;                      /* 0: exponential (Eq. 1); 1: Gaussian of equal FWHM */
    double e_res;                              /* adaptive sampling: finest step in e (E_RES) */
    int32_t np_max;                            /* adaptive sampling: samples above threshold wanted (NP_MAX) */
    int32_t estimator;                         /* 0: the fixed grid; 1: adaptive sampling around the maximum */
    int32_t refit_bad, pad2;                   /* 1: fit the bad fits again after the whole catalogue */
    double pos_step_arcsec;                    /* position marginal: offset step */
    int32_t n_pos, pad3;                       /* position marginal: offsets per axis (1: position exact) */
} rlfo_params;

int rlfo_nest(void) { return RLFO_NEST; }
int rlfo_params_size(void) { return (int)sizeof(rlfo_params); }

/* Eq. 4: ln(alpha_med / arcsec) = ADD + ESP ln(S / uJy).  Returns arcsec. */
double rlfo_alpha_med(double flux_jy, double add, double esp)
{
    return exp(add + esp * log(flux_jy * 1.0e6));
}

/* |A^{-T} k|^2 with A the shear matrix of Eq. 2, inverted explicitly. */
static double sheared_k2(double ku, double kv, double e1, double e2)
{
    double a11 = 1.0 - e1, a12 = -e2, a21 = -e2, a22 = 1.0 + e1;
    double det = a11 * a22 - a12 * a21;
    /* inverse of A */
    double i11 = a22 / det, i12 = -a12 / det, i21 = -a21 / det, i22 = a11 / det;
    /* transpose of the inverse applied to k */
    double x = i11 * ku + i21 * kv;
    double y = i12 * ku + i22 * kv;
    return x * x + y * y;
}

/*
 * The Eq. 1 brightness factor; k in wavelengths.
 *   profile 0, exponential disc: (1 + 4 pi^2 alpha^2 |A^{-T} k|^2)^{-3/2}
 *   profile 1, Gaussian: exp(-2 pi^2 sigma^2 |A^{-T} k|^2), the transform of
 *     exp(-r^2 / (2 sigma^2)), with sigma = alpha sqrt(ln 2 / 2) so that its FWHM,
 *     2 sigma sqrt(2 ln 2), equals the exponential's 2 alpha ln 2 (footnote to Sec. 2.2)
 */
double rlfo_shape(double ku, double kv, double alpha_rad, double e1, double e2, int profile)
{
    double k2 = sheared_k2(ku, kv, e1, e2);
    if (profile == 1) {
        double sigma2 = alpha_rad * alpha_rad * log(2.0) / 2.0;
        return exp(-2.0 * RLFO_PI * RLFO_PI * sigma2 * k2);
    }
    return pow(1.0 + 4.0 * RLFO_PI * RLFO_PI * alpha_rad * alpha_rad * k2, -1.5);
}

/* n - 1 = sqrt(1 - l^2 - m^2) - 1, written without cancellation */
static double n_minus_1(double l, double m)
{
    double r2 = l * l + m * m;
    return -r2 / (1.0 + sqrt(1.0 - r2));
}

/* Eq. 1: visibility of one source at baseline (u, v, w) metres and frequency freq. */
void rlfo_model_vis(double u, double v, double w, double freq, double l, double m,
                    double flux_jy, double alpha_rad, double e1, double e2,
                    double beta, double nu_ref, int profile, double *re, double *im)
{
    double s = freq / RLFO_C;
    double ku = u * s, kv = v * s, kw = w * s;
    double amp = pow(freq / nu_ref, beta) * flux_jy * rlfo_shape(ku, kv, alpha_rad, e1, e2, profile);
    double ph = 2.0 * RLFO_PI * (ku * l + kv * m + kw * n_minus_1(l, m));
    *re = amp * cos(ph);
    *im = amp * sin(ph);
}

/*
 * Sky model (Sec. 2.2): V[r, c] = sum_j Eq.1_j(u_r, v_r, w_r, nu_c).
 * rows: optional list of row indices (NULL = every row); out is [n_out][n_chan][2];
 * abs_out (optional) receives sum_j |term_j| per output, the scale of a
 * cancellation-aware tolerance.
 */
void rlfo_sky_model(int64_t n_rows, int32_t n_chan, const double *u, const double *v,
                    const double *w, const double *freq, const int64_t *rows, int64_t n_out,
                    int32_t n_src, const double *l, const double *m, const double *flux,
                    const double *alpha_rad, const double *e1, const double *e2,
                    double beta, double nu_ref, int profile, double *out, double *abs_out, int n_threads)
{
    if (!rows) n_out = n_rows;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t o = 0; o < n_out; ++o) {
        int64_t r = rows ? rows[o] : o;
        for (int32_t c = 0; c < n_chan; ++c) {
            double sr = 0.0, si = 0.0, sa = 0.0;
            for (int32_t j = 0; j < n_src; ++j) {
                double re, im;
                rlfo_model_vis(u[r], v[r], w[r], freq[c], l[j], m[j], flux[j], alpha_rad[j],
                               e1[j], e2[j], beta, nu_ref, profile, &re, &im);
                sr += re;
                si += im;
                sa += sqrt(re * re + im * im);
            }
            out[(o * n_chan + c) * 2 + 0] = sr;
            out[(o * n_chan + c) * 2 + 1] = si;
            if (abs_out) abs_out[o * n_chan + c] = sa;
        }
    }
}

/*
 * Data visibilities of a synthetic observation: the same sum of Eq. 1 over the
 * catalogue as rlfo_sky_model, used only to make test inputs (the "observed" sky
 * at the true shapes), arranged so that 1e11-term observations take minutes:
 *   - per (row, source): the phase argument phi = u l + v m + w (n - 1) in metres,
 *     the sheared baseline A^{-T} (u, v) (Eq. 2 inverted as in sheared_k2), and
 *     exp(2 pi i phi s_0) from the fractional cycles of phi s_0;
 *   - per channel: the phase factor of channel c + 1 is that of channel c times
 *     exp(2 pi i phi ds) when the channels are uniformly spaced (s_c = s_0 + c ds
 *     to 1e-12 relative; else each channel's factor is computed directly), and the
 *     exponential profile's (1 + x)^{-3/2} is 1 / ((1 + x) sqrt(1 + x)).
 * The result agrees with rlfo_sky_model to about 1e-14 of the summed moduli.
 * out is [n_rows][n_chan][2] doubles, overwritten.
 */
void rlfo_simulate_vis(int64_t n_rows, int32_t n_chan, const double *u, const double *v, const double *w,
                       const double *freq, int32_t n_src, const double *l, const double *m,
                       const double *flux, const double *alpha_rad, const double *e1, const double *e2,
                       double beta, double nu_ref, int profile, double *out, int n_threads)
{
    double *s = malloc(sizeof(double) * n_chan), *spec = malloc(sizeof(double) * n_chan);
    double *tab = malloc(sizeof(double) * 9 * (n_src > 0 ? n_src : 1));
    if (!s || !spec || !tab) { free(s); free(spec); free(tab); return; }
    for (int32_t c = 0; c < n_chan; ++c) {
        s[c] = freq[c] / RLFO_C;
        spec[c] = pow(freq[c] / nu_ref, beta);
    }
    const double ds = n_chan > 1 ? s[1] - s[0] : 0.0;
    int uniform = 1;
    for (int32_t c = 0; c < n_chan; ++c)
        if (fabs(s[c] - (s[0] + c * ds)) > 1e-12 * s[c]) uniform = 0;
    for (int32_t j = 0; j < n_src; ++j) {
        double *t = tab + 9 * j;
        double a11 = 1.0 - e1[j], a12 = -e2[j], a21 = -e2[j], a22 = 1.0 + e1[j];
        double det = a11 * a22 - a12 * a21;
        t[0] = a22 / det; t[1] = -a12 / det; t[2] = -a21 / det; t[3] = a11 / det;
        t[4] = profile == 1 ? 2.0 * RLFO_PI * RLFO_PI * alpha_rad[j] * alpha_rad[j] * log(2.0) / 2.0
                            : 4.0 * RLFO_PI * RLFO_PI * alpha_rad[j] * alpha_rad[j];
        t[5] = n_minus_1(l[j], m[j]);
        t[6] = flux[j];
        t[7] = l[j];
        t[8] = m[j];
    }
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t r = 0; r < n_rows; ++r) {
        double *o = out + r * n_chan * 2;
        for (int32_t c = 0; c < 2 * n_chan; ++c) o[c] = 0.0;
        for (int32_t j = 0; j < n_src; ++j) {
            const double *t = tab + 9 * j;
            double x = t[0] * u[r] + t[2] * v[r];
            double y = t[1] * u[r] + t[3] * v[r];
            double q = t[4] * (x * x + y * y);
            double phi = u[r] * t[7] + v[r] * t[8] + w[r] * t[5];
            double f0 = phi * s[0];
            f0 -= rint(f0);
            double zr = cos(2.0 * RLFO_PI * f0), zi = sin(2.0 * RLFO_PI * f0), sr = 1.0, si = 0.0;
            if (uniform && n_chan > 1) {
                double fd = phi * ds;
                fd -= rint(fd);
                sr = cos(2.0 * RLFO_PI * fd);
                si = sin(2.0 * RLFO_PI * fd);
            }
            for (int32_t c = 0; c < n_chan; ++c) {
                if (!uniform && c > 0) {
                    double fc = phi * s[c];
                    fc -= rint(fc);
                    zr = cos(2.0 * RLFO_PI * fc);
                    zi = sin(2.0 * RLFO_PI * fc);
                }
                double qc = q * s[c] * s[c];
                double br;
                if (profile == 1) {
                    br = exp(-qc);
                } else {
                    double xp = 1.0 + qc;
                    br = 1.0 / (xp * sqrt(xp));
                }
                double amp = t[6] * spec[c] * br;
                o[2 * c] += amp * zr;
                o[2 * c + 1] += amp * zi;
                if (uniform) {
                    double nr = zr * sr - zi * si;
                    zi = zr * si + zi * sr;
                    zr = nr;
                }
            }
        }
    }
    free(s);
    free(spec);
    free(tab);
}

/*
 * Facet of one source (Sec. 2.3).
 *   residual   R = D - V_sky + model_i     (every source but i removed)
 *   shifted    x = R * exp(-2 pi i (u l + v m + w (n - 1)))
 *   cell       (iu, iv) = floor(k / du) + N/2 on an N x N window centred on the
 *              origin; visibilities outside the window are dropped (reading).
 * acc is [4][N*N]: sum Re x, sum Im x, count, sum of the spectral factor
 * (nu/nu_ref)^beta; cell index iv * N + iu.  abs_acc (optional) is sum |x|.
 * The sky model is read either as complex64 (sky_f) or complex128 (sky_d).
 * The source model added back uses the source's current sky-model shape
 * (e1_cur, e2_cur) and scalelength alpha_sky_rad.
 */
void rlfo_extract_facet(int64_t n_rows, int32_t n_chan, const double *u, const double *v,
                        const double *w, const double *freq, const float *data,
                        const float *sky_f, const double *sky_d,
                        double l, double m, double flux, double alpha_sky_rad,
                        double e1_cur, double e2_cur, double beta, double nu_ref, int profile,
                        double du, int32_t facet_n, double *acc, double *abs_acc)
{
    const int64_t nc = (int64_t)facet_n * facet_n;
    memset(acc, 0, sizeof(double) * 4 * nc);
    if (abs_acc) memset(abs_acc, 0, sizeof(double) * nc);
    const double n1 = n_minus_1(l, m);
    for (int64_t r = 0; r < n_rows; ++r) {
        for (int32_t c = 0; c < n_chan; ++c) {
            double s = freq[c] / RLFO_C;
            double ku = u[r] * s, kv = v[r] * s, kw = w[r] * s;
            double fu = floor(ku / du), fv = floor(kv / du);
            if (fu < -facet_n / 2 || fu >= facet_n / 2 || fv < -facet_n / 2 || fv >= facet_n / 2)
                continue;
            int64_t iu = (int64_t)fu + facet_n / 2, iv = (int64_t)fv + facet_n / 2;
            int64_t idx = (r * n_chan + c) * 2;
            double skr = sky_f ? (double)sky_f[idx] : sky_d[idx];
            double ski = sky_f ? (double)sky_f[idx + 1] : sky_d[idx + 1];
            double mr, mi;
            rlfo_model_vis(u[r], v[r], w[r], freq[c], l, m, flux, alpha_sky_rad, e1_cur, e2_cur,
                           beta, nu_ref, profile, &mr, &mi);
            double rr = (double)data[idx] - skr + mr;
            double ri = (double)data[idx + 1] - ski + mi;
            double ph = -2.0 * RLFO_PI * (ku * l + kv * m + kw * n1);
            double cr = cos(ph), ci = sin(ph);
            double xr = rr * cr - ri * ci;
            double xi = rr * ci + ri * cr;
            int64_t cell = iv * facet_n + iu;
            acc[0 * nc + cell] += xr;
            acc[1 * nc + cell] += xi;
            acc[2 * nc + cell] += 1.0;
            acc[3 * nc + cell] += pow(freq[c] / nu_ref, beta);
            if (abs_acc) abs_acc[cell] += sqrt(xr * xr + xi * xi);
        }
    }
}

/* ln erfc(x) + x^2 for x > 25: the asymptotic series of Abramowitz & Stegun 7.1.23 */
static double log_erfc_scaled_tail(double x)
{
    double t = 1.0 / (2.0 * x * x);
    /* 1 - 1/(2x^2) + 3/(2x^2)^2 - 15/(2x^2)^3 + 105/(2x^2)^4 */
    double series = 1.0 - t + 3.0 * t * t - 15.0 * t * t * t + 105.0 * t * t * t * t;
    return -log(x * sqrt(RLFO_PI)) + log(series);
}

/*
 * Flux-marginalised log-likelihood (Sec. 2.4): chi^2 = C - 2 S b + S^2 a and a
 * uniform flux prior give
 *   S in [0, inf):  -C/2 + b^2/(2a) + ln sqrt(pi/(2a)) + ln erfc(-b/sqrt(2a))
 *   S on the line:  -C/2 + b^2/(2a) + ln sqrt(2 pi/a)
 * When x = -b/sqrt(2a) > 25 the b^2/(2a) = x^2 term cancels the leading -x^2 of
 * ln erfc(x); that cancellation is done analytically.
 */
double rlfo_flux_marginal(double a, double b, double cc, int flux_prior)
{
    if (flux_prior == 1)
        return -0.5 * cc + b * b / (2.0 * a) + 0.5 * log(2.0 * RLFO_PI / a);
    double x = -b / sqrt(2.0 * a);
    if (x > 25.0)
        return -0.5 * cc + 0.5 * log(RLFO_PI / (2.0 * a)) + log_erfc_scaled_tail(x);
    return -0.5 * cc + b * b / (2.0 * a) + 0.5 * log(RLFO_PI / (2.0 * a)) + log(erfc(x));
}

double rlfo_grid_e(const rlfo_params *p, int k)
{
    return -p->e_max + k * (2.0 * p->e_max / (p->n_e - 1));
}

/* scalelength nodes with quadratic spacing on [RMIN, RMAX] (Sec. 2.4, Sec. 4.2); arcsec */
double rlfo_grid_alpha(const rlfo_params *p, int k)
{
    double t = (p->n_alpha > 1) ? (double)k / (p->n_alpha - 1) : 0.0;
    return p->r_min_arcsec + (p->r_max_arcsec - p->r_min_arcsec) * t * t;
}

typedef struct {
    int ncell;
    double cc;
    double *cu, *cv, *cw, *cs, *cd, *ci;
    double *cr;   /* position marginal: [n_pos^2][ncell] Re(D_c exp(-2 pi i k_c.x_j)), else NULL */
} rlfo_cells;

static void cells_of_facet(const double *acc, double du, const rlfo_params *p, rlfo_cells *C)
{
    const int N = p->facet_n;
    const int64_t nc = (int64_t)N * N;
    const double sig2 = p->sigma_jy * p->sigma_jy;
    C->cu = malloc(sizeof(double) * nc);
    C->cv = malloc(sizeof(double) * nc);
    C->cw = malloc(sizeof(double) * nc);
    C->cs = malloc(sizeof(double) * nc);
    C->cd = malloc(sizeof(double) * nc);
    C->ci = malloc(sizeof(double) * nc);
    C->ncell = 0;
    C->cc = 0.0;
    for (int iv = 0; iv < N; ++iv)
        for (int iu = 0; iu < N; ++iu) {
            int64_t cell = (int64_t)iv * N + iu;
            double n = acc[2 * nc + cell];
            if (n <= 0.0) continue;
            double dr = acc[cell] / n, di = acc[nc + cell] / n;
            int c = C->ncell++;
            C->cu[c] = (iu - N / 2 + 0.5) * du;
            C->cv[c] = (iv - N / 2 + 0.5) * du;
            C->cw[c] = n / sig2;
            C->cs[c] = acc[3 * nc + cell] / n;
            C->cd[c] = dr;
            C->ci[c] = di;
            C->cc += C->cw[c] * (dr * dr + di * di);
        }
    /* the data of every cell seen from each position offset x_j (Sec. 2.4): an offset
       source's model carries exp(+2 pi i k.x_j), so its b uses Re(D exp(-2 pi i k.x_j)) */
    C->cr = NULL;
    if (p->n_pos > 1 && p->n_pos <= 7 && p->n_pos % 2 == 1) {
        const int np = p->n_pos, nj = np * np;
        const double step = p->pos_step_arcsec * RLFO_ARCSEC;
        C->cr = malloc(sizeof(double) * nj * (C->ncell > 0 ? C->ncell : 1));
        for (int j = 0; j < nj; ++j) {
            double dl = (j / np - (np - 1) / 2) * step, dm = (j % np - (np - 1) / 2) * step;
            for (int c = 0; c < C->ncell; ++c) {
                double th = 2.0 * RLFO_PI * (C->cu[c] * dl + C->cv[c] * dm);
                C->cr[(int64_t)j * C->ncell + c] = C->cd[c] * cos(th) + C->ci[c] * sin(th);
            }
        }
    }
}

static void free_cells(rlfo_cells *C)
{
    free(C->cu); free(C->cv); free(C->cw); free(C->cs); free(C->cd); free(C->ci); free(C->cr);
}


/*
 * Flux-marginalised log-likelihood of one (e, alpha) point over a facet's cells
 * (Sec. 2.4): a = sum w s^2 M^2, b = sum w s M Re D.  With n_pos > 1 the source
 * position is marginalised too, with a uniform prior over an n_pos x n_pos grid of
 * offsets x0 (step pos_step_arcsec, centred on the catalogue position; n_pos odd,
 * at most 7, else NaN): an offset
 * source's facet model carries exp(+2 pi i k.x0), so a and C are unchanged and
 * b(x0) = sum w s M Re(D exp(-2 pi i k.x0)); the marginal is the mean of
 * exp(logL(x0)) over the offsets, and *b_out is b at the best offset.
 */
static double like_point(const rlfo_cells *C, double e1, double e2, double al, const rlfo_params *p,
                         double *a_out, double *b_out)
{
    double a = 0.0;
    if (p->n_pos <= 1) {
        double b = 0.0;
        for (int c = 0; c < C->ncell; ++c) {
            double M = rlfo_shape(C->cu[c], C->cv[c], al, e1, e2, p->profile);
            a += C->cw[c] * C->cs[c] * C->cs[c] * M * M;
            b += C->cw[c] * C->cs[c] * M * C->cd[c];
        }
        *a_out = a;
        *b_out = b;
        return rlfo_flux_marginal(a, b, C->cc, p->flux_prior);
    }
    const int np = p->n_pos, nj = np * np;
    if (np > 7 || np % 2 == 0) {   /* odd grids up to 7 x 7 only */
        *a_out = *b_out = NAN;
        return NAN;
    }
    double bj[64];
    for (int j = 0; j < nj; ++j) bj[j] = 0.0;
    for (int c = 0; c < C->ncell; ++c) {
        double M = rlfo_shape(C->cu[c], C->cv[c], al, e1, e2, p->profile);
        a += C->cw[c] * C->cs[c] * C->cs[c] * M * M;
        double wsm = C->cw[c] * C->cs[c] * M;
        for (int j = 0; j < nj; ++j) bj[j] += wsm * C->cr[(int64_t)j * C->ncell + c];
    }
    double lmax = -INFINITY;
    int jbest = 0;
    double lj[64];
    for (int j = 0; j < nj; ++j) {
        lj[j] = rlfo_flux_marginal(a, bj[j], C->cc, p->flux_prior);
        if (lj[j] > lmax) {
            lmax = lj[j];
            jbest = j;
        }
    }
    double s = 0.0;
    for (int j = 0; j < nj; ++j) s += exp(lj[j] - lmax);
    *a_out = a;
    *b_out = bj[jbest];
    return lmax + log(s / nj);
}

/*
 * Likelihood grid of one facet (Sec. 2.4) on e1, e2 in {-e_max .. e_max} (n_e
 * nodes, |e| < 1 only) x alpha nodes.  loglike/a_out/b_out are
 * [n_e][n_e][n_alpha] (e1 outer, alpha inner); invalid points get -inf, 0, 0.
 * The facet model of a cell is S * s_c * shape(k_c) at the cell centre, w = 0.
 * Returns the number of non-empty cells.
 */
int rlfo_like_grid(const double *acc, double du, const rlfo_params *p,
                   double *loglike, double *a_out, double *b_out)
{
    const int ne = p->n_e, na = p->n_alpha;
    /* cell averages and weights: D_c = mean x, s_c = mean spectral factor, w_c = n_c / sigma^2 */
    rlfo_cells C;
    cells_of_facet(acc, du, p, &C);
    for (int i1 = 0; i1 < ne; ++i1)
        for (int i2 = 0; i2 < ne; ++i2) {
            double e1 = rlfo_grid_e(p, i1), e2 = rlfo_grid_e(p, i2);
            int valid = (e1 * e1 + e2 * e2 < 1.0);
            for (int k = 0; k < na; ++k) {
                int64_t g = ((int64_t)i1 * ne + i2) * na + k;
                if (!valid || C.ncell == 0) {
                    loglike[g] = -INFINITY;
                    a_out[g] = 0.0;
                    b_out[g] = 0.0;
                    continue;
                }
                loglike[g] = like_point(&C, e1, e2, rlfo_grid_alpha(p, k) * RLFO_ARCSEC, p, &a_out[g], &b_out[g]);
            }
        }
    int ncell = C.ncell;
    free_cells(&C);
    return ncell;
}

/* trapezoid weight times the log-normal scalelength prior (mean from Eq. 4, sigma R_STD) */
double rlfo_alpha_weight(const rlfo_params *p, double flux_cat, int k)
{
    const int na = p->n_alpha;
    double ak = rlfo_grid_alpha(p, k);
    double q;
    if (na == 1) q = 1.0;
    else if (k == 0) q = 0.5 * (rlfo_grid_alpha(p, 1) - ak);
    else if (k == na - 1) q = 0.5 * (ak - rlfo_grid_alpha(p, na - 2));
    else q = 0.5 * (rlfo_grid_alpha(p, k + 1) - rlfo_grid_alpha(p, k - 1));
    double mu = p->add + p->esp * log(flux_cat * 1.0e6);
    double z = (log(ak) - mu) / p->r_std;
    return q * exp(-0.5 * z * z) / (ak * p->r_std * sqrt(2.0 * RLFO_PI));
}

/*
 * Estimate from a likelihood grid (Sec. 2.4): marginalise alpha numerically,
 * keep the e points whose marginal is at least thresh_frac of its maximum, and
 * return their likelihood-weighted mean and standard deviation; the bad-fit cut
 * of Sec. 4.1 sets the flag.  Le_out (optional, [n_e*n_e]) receives the
 * alpha-marginal L(e) relative to exp(max logL).
 */
void rlfo_estimate(const double *loglike, const double *a_out, const double *b_out,
                   double flux_cat, int ncell, const rlfo_params *p, double *est, double *Le_out)
{
    const int ne = p->n_e, na = p->n_alpha;
    double lmax = -INFINITY;
    for (int64_t g = 0; g < (int64_t)ne * ne * na; ++g)
        if (loglike[g] > lmax) lmax = loglike[g];
    double *qp = malloc(sizeof(double) * na);
    for (int k = 0; k < na; ++k) qp[k] = rlfo_alpha_weight(p, flux_cat, k);
    double mu = p->add + p->esp * log(flux_cat * 1.0e6);

    /* marginal over alpha: L(e) = sum_k q_k p(alpha_k) exp(logL(e, alpha_k) - lmax) */
    double *Le = malloc(sizeof(double) * ne * ne);
    double *Ae = malloc(sizeof(double) * ne * ne);
    double Lmax = 0.0;
    for (int e = 0; e < ne * ne; ++e) {
        double s = 0.0, sa = 0.0;
        for (int k = 0; k < na; ++k) {
            double lg = loglike[(int64_t)e * na + k];
            if (lg == -INFINITY) continue;
            double t = qp[k] * exp(lg - lmax);
            s += t;
            sa += t * rlfo_grid_alpha(p, k);
        }
        Le[e] = s;
        Ae[e] = sa;
        if (s > Lmax) Lmax = s;
        if (Le_out) Le_out[e] = s;
    }

    /* moments over the points above thresh_frac * Lmax, and over all points */
    double W = 0, m1 = 0, m2 = 0, WA = 0, Ws = 0, s1 = 0, s2 = 0;
    double margin = INFINITY;
    for (int e = 0; e < ne * ne; ++e) {
        if (!(Le[e] > 0.0)) continue;
        double e1 = rlfo_grid_e(p, e / ne), e2 = rlfo_grid_e(p, e % ne);
        Ws += Le[e];
        s1 += Le[e] * e1;
        s2 += Le[e] * e2;
        double dm = fabs(log(Le[e] / Lmax) - log(p->thresh_frac));
        if (dm < margin) margin = dm;
        if (Le[e] >= p->thresh_frac * Lmax) {
            W += Le[e];
            m1 += Le[e] * e1;
            m2 += Le[e] * e2;
            WA += Ae[e];
        }
    }
    double e1m = 0, e2m = 0, c11 = 0, c22 = 0, c12 = 0, am = 0;
    if (W > 0) {
        e1m = m1 / W;
        e2m = m2 / W;
        am = WA / W;
        for (int e = 0; e < ne * ne; ++e) {
            if (!(Le[e] > 0.0) || Le[e] < p->thresh_frac * Lmax) continue;
            double d1 = rlfo_grid_e(p, e / ne) - e1m, d2 = rlfo_grid_e(p, e % ne) - e2m;
            c11 += Le[e] * d1 * d1;
            c22 += Le[e] * d2 * d2;
            c12 += Le[e] * d1 * d2;
        }
        c11 /= W;
        c22 /= W;
        c12 /= W;
    }
    /* maximum a posteriori grid point: logL + ln p(alpha); ties -> lowest flat index */
    int64_t gmap = -1;
    double best = -INFINITY;
    for (int64_t g = 0; g < (int64_t)ne * ne * na; ++g) {
        if (loglike[g] == -INFINITY) continue;
        double ak = rlfo_grid_alpha(p, (int)(g % na));
        double z = (log(ak) - mu) / p->r_std;
        double lp = loglike[g] - 0.5 * z * z - log(ak);
        if (lp > best) {
            best = lp;
            gmap = g;
        }
    }
    double s1d = sqrt(c11), s2d = sqrt(c22);
    double det = c11 * c22 - c12 * c12;
    double sdet = det > 0 ? sqrt(det) : 0.0;
    int bad = (W <= 0) || (s1d <= p->var_sigma_min) || (s2d <= p->var_sigma_min) ||
              (sdet <= p->var_det_min);
    est[RLFO_E1] = e1m;
    est[RLFO_E2] = e2m;
    est[RLFO_SIG1] = s1d;
    est[RLFO_SIG2] = s2d;
    est[RLFO_ALPHA] = am;
    est[RLFO_FLUX] = (gmap >= 0 && a_out[gmap] > 0) ? b_out[gmap] / a_out[gmap] : 0.0;
    est[RLFO_FLAG] = bad ? 1.0 : 0.0;
    est[RLFO_E1_SMOOTH] = Ws > 0 ? s1 / Ws : 0.0;
    est[RLFO_E2_SMOOTH] = Ws > 0 ? s2 / Ws : 0.0;
    est[RLFO_LOGL_MAX] = lmax;
    est[RLFO_THRESH_MARGIN] = margin;
    est[RLFO_MAP_INDEX] = (double)gmap;
    est[RLFO_NC] = (double)ncell;
    est[RLFO_LEVELS] = 0.0;
    est[RLFO_STEP] = 2.0 * p->e_max / (ne - 1);
    est[RLFO_NKEPT] = 0.0;
    for (int e = 0; e < ne * ne; ++e)
        if (Le[e] > 0.0 && Le[e] >= p->thresh_frac * Lmax) est[RLFO_NKEPT] += 1.0;
    free(qp); free(Le); free(Ae);
}

/*
 * Adaptive sampling of the alpha-marginal likelihood L(e) around its maximum
 * (Sec. 2.4), read as successive lattices: level 0 is the fixed grid (step h0 =
 * 2 e_max / (n_e - 1)); while fewer than np_max samples lie at or above
 * thresh_frac of the level's maximum and the step is above e_res, the step is
 * halved and L(e) is sampled at every multiple of the new step in the box spanned
 * by the kept samples, widened by the previous step (points with |e| >= 1
 * skipped; at most 17 per component, centred on the level's MAP sample).  The
 * estimate is the last level's: the same threshold moments, MAP flux and bad-fit
 * cut as the grid estimate, over its samples.  est[RLFO_LEVELS] = refinements
 * made, est[RLFO_STEP] = last step, est[RLFO_NKEPT] = samples kept.
 */
/* loglike, a, b of every (sample, alpha node) pair: [np][n_alpha] */
static void sample_likelihood(const rlfo_cells *C, const double *e1s, const double *e2s, int np,
                              const rlfo_params *p, double *loglike, double *a_out, double *b_out)
{
    const int na = p->n_alpha;
    for (int i = 0; i < np; ++i)
        for (int k = 0; k < na; ++k) {
            int64_t g = (int64_t)i * na + k;
            if (!(e1s[i] * e1s[i] + e2s[i] * e2s[i] < 1.0) || C->ncell == 0) {
                loglike[g] = -INFINITY;
                a_out[g] = b_out[g] = 0.0;
                continue;
            }
            loglike[g] = like_point(C, e1s[i], e2s[i], rlfo_grid_alpha(p, k) * RLFO_ARCSEC, p, &a_out[g],
                                    &b_out[g]);
        }
}

/*
 * The estimate of Sec. 2.4 over an explicit list of e samples (the grid estimate
 * restated for any sample set): alpha marginal, threshold moments, MAP sample
 * (logL + ln p(alpha), ties to the lowest (sample, alpha) index), bad-fit cut.
 * Also returns the number of kept samples, the box they span and the MAP sample.
 */
static void estimate_samples(const double *e1s, const double *e2s, int np, const double *loglike,
                             const double *a_out, const double *b_out, double flux_cat, int ncell,
                             const rlfo_params *p, double *est, int *n_kept, double box[4], int *map_sample)
{
    const int na = p->n_alpha;
    double lmax = -INFINITY;
    for (int64_t g = 0; g < (int64_t)np * na; ++g)
        if (loglike[g] > lmax) lmax = loglike[g];
    double mu = p->add + p->esp * log(flux_cat * 1.0e6);
    double *Le = malloc(sizeof(double) * np), *Ae = malloc(sizeof(double) * np);
    double Lmax = 0.0;
    for (int i = 0; i < np; ++i) {
        double sL = 0.0, sA = 0.0;
        for (int k = 0; k < na; ++k) {
            double lg = loglike[(int64_t)i * na + k];
            if (lg == -INFINITY) continue;
            double t = rlfo_alpha_weight(p, flux_cat, k) * exp(lg - lmax);
            sL += t;
            sA += t * rlfo_grid_alpha(p, k);
        }
        Le[i] = sL;
        Ae[i] = sA;
        if (sL > Lmax) Lmax = sL;
    }
    double W = 0, m1 = 0, m2 = 0, WA = 0, Ws = 0, s1 = 0, s2 = 0, margin = INFINITY;
    int kept = 0;
    box[0] = box[2] = INFINITY;
    box[1] = box[3] = -INFINITY;
    for (int i = 0; i < np; ++i) {
        if (!(Le[i] > 0.0)) continue;
        Ws += Le[i];
        s1 += Le[i] * e1s[i];
        s2 += Le[i] * e2s[i];
        double dm = fabs(log(Le[i] / Lmax) - log(p->thresh_frac));
        if (dm < margin) margin = dm;
        if (Le[i] >= p->thresh_frac * Lmax) {
            ++kept;
            W += Le[i];
            m1 += Le[i] * e1s[i];
            m2 += Le[i] * e2s[i];
            WA += Ae[i];
            if (e1s[i] < box[0]) box[0] = e1s[i];
            if (e1s[i] > box[1]) box[1] = e1s[i];
            if (e2s[i] < box[2]) box[2] = e2s[i];
            if (e2s[i] > box[3]) box[3] = e2s[i];
        }
    }
    double e1m = 0, e2m = 0, c11 = 0, c22 = 0, c12 = 0, am = 0;
    if (W > 0) {
        e1m = m1 / W;
        e2m = m2 / W;
        am = WA / W;
        for (int i = 0; i < np; ++i) {
            if (!(Le[i] > 0.0) || Le[i] < p->thresh_frac * Lmax) continue;
            double d1 = e1s[i] - e1m, d2 = e2s[i] - e2m;
            c11 += Le[i] * d1 * d1;
            c22 += Le[i] * d2 * d2;
            c12 += Le[i] * d1 * d2;
        }
        c11 /= W;
        c22 /= W;
        c12 /= W;
    }
    int64_t gmap = -1;
    double best = -INFINITY;
    for (int64_t g = 0; g < (int64_t)np * na; ++g) {
        if (loglike[g] == -INFINITY) continue;
        double ak = rlfo_grid_alpha(p, (int)(g % na));
        double z = (log(ak) - mu) / p->r_std;
        double lp = loglike[g] - 0.5 * z * z - log(ak);
        if (lp > best) {
            best = lp;
            gmap = g;
        }
    }
    double s1d = sqrt(c11), s2d = sqrt(c22);
    double det = c11 * c22 - c12 * c12;
    double sdet = det > 0 ? sqrt(det) : 0.0;
    int bad = (W <= 0) || (s1d <= p->var_sigma_min) || (s2d <= p->var_sigma_min) || (sdet <= p->var_det_min);
    est[RLFO_E1] = e1m;
    est[RLFO_E2] = e2m;
    est[RLFO_SIG1] = s1d;
    est[RLFO_SIG2] = s2d;
    est[RLFO_ALPHA] = am;
    est[RLFO_FLUX] = (gmap >= 0 && a_out[gmap] > 0) ? b_out[gmap] / a_out[gmap] : 0.0;
    est[RLFO_FLAG] = bad ? 1.0 : 0.0;
    est[RLFO_E1_SMOOTH] = Ws > 0 ? s1 / Ws : 0.0;
    est[RLFO_E2_SMOOTH] = Ws > 0 ? s2 / Ws : 0.0;
    est[RLFO_LOGL_MAX] = lmax;
    est[RLFO_THRESH_MARGIN] = margin;
    est[RLFO_MAP_INDEX] = (double)gmap;
    est[RLFO_NC] = (double)ncell;
    *n_kept = kept;
    *map_sample = gmap >= 0 ? (int)(gmap / na) : -1;
    free(Le);
    free(Ae);
}

void rlfo_fit_facet_adaptive(const double *acc, double du, double flux_cat, const rlfo_params *p, double *est)
{
    const int ne = p->n_e, na = p->n_alpha;
    const int kMaxSide = 17;
    rlfo_cells C;
    cells_of_facet(acc, du, p, &C);
    /* level 0: the fixed grid, samples in grid order (e1 outer, e2 inner) */
    int np = ne * ne;
    int cap = kMaxSide * kMaxSide > np ? kMaxSide * kMaxSide : np;
    double *e1s = malloc(sizeof(double) * cap), *e2s = malloc(sizeof(double) * cap);
    double *lg = malloc(sizeof(double) * cap * na), *ga = malloc(sizeof(double) * cap * na);
    double *gb = malloc(sizeof(double) * cap * na);
    for (int i1 = 0; i1 < ne; ++i1)
        for (int i2 = 0; i2 < ne; ++i2) {
            e1s[i1 * ne + i2] = rlfo_grid_e(p, i1);
            e2s[i1 * ne + i2] = rlfo_grid_e(p, i2);
        }
    double h = 2.0 * p->e_max / (ne - 1);
    int level = 0, kept = 0, map_i = -1;
    double box[4];
    for (;;) {
        sample_likelihood(&C, e1s, e2s, np, p, lg, ga, gb);
        estimate_samples(e1s, e2s, np, lg, ga, gb, flux_cat, C.ncell, p, est, &kept, box, &map_i);
        if (p->estimator != 1 || kept >= p->np_max || h <= p->e_res || map_i < 0) break;
        /* the next lattice: multiples of h/2 in the kept box widened by h */
        double hn = 0.5 * h;
        int lo[2], hi[2];
        double cen[2] = {e1s[map_i], e2s[map_i]};
        for (int d = 0; d < 2; ++d) {
            lo[d] = (int)ceil((box[2 * d] - h) / hn - 1e-9);
            hi[d] = (int)floor((box[2 * d + 1] + h) / hn + 1e-9);
            if (hi[d] - lo[d] + 1 > kMaxSide) {
                int c = (int)llround(cen[d] / hn);
                lo[d] = c - kMaxSide / 2;
                hi[d] = c + kMaxSide / 2;
            }
        }
        np = 0;
        for (int i1 = lo[0]; i1 <= hi[0]; ++i1)
            for (int i2 = lo[1]; i2 <= hi[1]; ++i2) {
                double a1 = i1 * hn, a2 = i2 * hn;
                if (!(a1 * a1 + a2 * a2 < 1.0)) continue;
                e1s[np] = a1;
                e2s[np] = a2;
                ++np;
            }
        h = hn;
        ++level;
    }
    est[RLFO_LEVELS] = level;
    est[RLFO_STEP] = h;
    est[RLFO_NKEPT] = kept;
    free(e1s); free(e2s); free(lg); free(ga); free(gb);
    free_cells(&C);
}

/* likelihood grid followed by the estimate */
void rlfo_fit_facet(const double *acc, double du, double flux_cat, const rlfo_params *p,
                    double *loglike, double *a_out, double *b_out, double *est)
{
    int ncell = rlfo_like_grid(acc, du, p, loglike, a_out, b_out);
    rlfo_estimate(loglike, a_out, b_out, flux_cat, ncell, p, est, NULL);
}

/* facet cell size du = 1 / (K alpha) in wavelengths (Sec. 2.3); alpha in arcsec */
double rlfo_facet_du(double flux_jy, double alpha_cat_arcsec, const rlfo_params *p)
{
    double a = alpha_cat_arcsec > 0 ? alpha_cat_arcsec : rlfo_alpha_med(flux_jy, p->add, p->esp);
    return 1.0 / (p->psf_nat * a * RLFO_ARCSEC);
}

/* One chunk of the chain: extract the listed sources' facets from the current sky
   model, fit them, and replace their shapes in the sky model (good fits, or all
   with update_mode 1). */
static void chunk_step(int64_t n_rows, int32_t n_chan, const double *u, const double *v, const double *w,
                       const double *freq, const float *data, const double *l, const double *m,
                       const double *flux, const double *alpha_cat_arcsec, const rlfo_params *p, double *est,
                       double *sky, const double *alpha_sky, double *e1c, double *e2c, const int *list, int cnt,
                       int n_threads)
{
    const int64_t nc = (int64_t)p->facet_n * p->facet_n;
    const int ng = p->n_e * p->n_e * p->n_alpha;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int t = 0; t < cnt; ++t) {
        int i = list[t];
        double *acc = malloc(sizeof(double) * 4 * nc);
        double *lg = malloc(sizeof(double) * ng * 3);
        double du = rlfo_facet_du(flux[i], alpha_cat_arcsec ? alpha_cat_arcsec[i] : 0.0, p);
        rlfo_extract_facet(n_rows, n_chan, u, v, w, freq, data, NULL, sky, l[i], m[i], flux[i],
                           alpha_sky[i], e1c[i], e2c[i], p->beta, p->nu_ref_hz, p->profile, du,
                           p->facet_n, acc, NULL);
        double *e = est + (int64_t)i * RLFO_NEST;
        if (p->estimator == 1)
            rlfo_fit_facet_adaptive(acc, du, flux[i], p, e);
        else
            rlfo_fit_facet(acc, du, flux[i], p, lg, lg + ng, lg + 2 * ng, e);
        free(acc);
        free(lg);
    }
    /* sky update: V += model_i(e_new) - model_i(e_cur) for the chunk */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t r = 0; r < n_rows; ++r)
        for (int32_t c = 0; c < n_chan; ++c)
            for (int t = 0; t < cnt; ++t) {
                int i = list[t];
                const double *e = est + (int64_t)i * RLFO_NEST;
                if (p->update_mode == 0 && e[RLFO_FLAG] != 0.0) continue;
                double nr, ni, orr, oi;
                rlfo_model_vis(u[r], v[r], w[r], freq[c], l[i], m[i], flux[i], alpha_sky[i],
                               e[RLFO_E1], e[RLFO_E2], p->beta, p->nu_ref_hz, p->profile, &nr, &ni);
                rlfo_model_vis(u[r], v[r], w[r], freq[c], l[i], m[i], flux[i], alpha_sky[i],
                               e1c[i], e2c[i], p->beta, p->nu_ref_hz, p->profile, &orr, &oi);
                sky[(r * n_chan + c) * 2 + 0] += nr - orr;
                sky[(r * n_chan + c) * 2 + 1] += ni - oi;
            }
    for (int t = 0; t < cnt; ++t) {
        int i = list[t];
        const double *e = est + (int64_t)i * RLFO_NEST;
        if (p->update_mode == 0 && e[RLFO_FLAG] != 0.0) continue;
        e1c[i] = e[RLFO_E1];
        e2c[i] = e[RLFO_E2];
    }
}

/*
 * Whole chain (Sec. 2): circular sky model, then for each chunk of sources in
 * catalogue order: extract every facet of the chunk from the current sky model,
 * fit them, and replace their shapes in the sky model (good fits only, or all
 * with update_mode 1).  chunk = 1 is the serial order; chunk = n_src extracts
 * everything from the initial model (Sec. 3.1 on chunked updates).
 * est is [n_src][RLFO_NEST]; sky_out (optional) receives the final sky model.
 */
int rlfo_pipeline(int64_t n_rows, int32_t n_chan, const double *u, const double *v,
                  const double *w, const double *freq, const float *data, int32_t n_src,
                  const double *l, const double *m, const double *flux,
                  const double *alpha_cat_arcsec, const rlfo_params *p, double *est,
                  double *sky_out, int n_threads)
{
    const int64_t nv = n_rows * n_chan;
    double *sky = malloc(sizeof(double) * nv * 2);
    double *alpha_sky = malloc(sizeof(double) * n_src);
    double *e1c = calloc(n_src, sizeof(double)), *e2c = calloc(n_src, sizeof(double));
    if (!sky || !alpha_sky || !e1c || !e2c) return 1;
    for (int j = 0; j < n_src; ++j) {
        double a = alpha_cat_arcsec && alpha_cat_arcsec[j] > 0 ? alpha_cat_arcsec[j]
                                                               : rlfo_alpha_med(flux[j], p->add, p->esp);
        alpha_sky[j] = a * RLFO_ARCSEC;
    }
    rlfo_sky_model(n_rows, n_chan, u, v, w, freq, NULL, 0, n_src, l, m, flux, alpha_sky, e1c, e2c,
                   p->beta, p->nu_ref_hz, p->profile, sky, NULL, n_threads);
    int chunk = p->chunk > 0 ? p->chunk : n_src;
    int *idx = malloc(sizeof(int) * n_src);
    if (!idx) return 1;
    for (int i = 0; i < n_src; ++i) idx[i] = i;
    for (int first = 0; first < n_src; first += chunk) {
        int cnt = (first + chunk <= n_src) ? chunk : n_src - first;
        chunk_step(n_rows, n_chan, u, v, w, freq, data, l, m, flux, alpha_cat_arcsec, p, est, sky, alpha_sky,
                   e1c, e2c, idx + first, cnt, n_threads);
    }
    /* the bad fits once more, against the sky model of every other measured shape
       (Sec. 2.4), in catalogue order and chunks of the same size */
    if (p->refit_bad) {
        int nb = 0;
        for (int i = 0; i < n_src; ++i)
            if (est[(int64_t)i * RLFO_NEST + RLFO_FLAG] != 0.0) idx[nb++] = i;
        for (int first = 0; first < nb; first += chunk) {
            int cnt = (first + chunk <= nb) ? chunk : nb - first;
            chunk_step(n_rows, n_chan, u, v, w, freq, data, l, m, flux, alpha_cat_arcsec, p, est, sky, alpha_sky,
                       e1c, e2c, idx + first, cnt, n_threads);
            for (int t = 0; t < cnt; ++t) est[(int64_t)idx[first + t] * RLFO_NEST + RLFO_REFIT] = 1.0;
        }
    }
    free(idx);
    if (sky_out) memcpy(sky_out, sky, sizeof(double) * nv * 2);
    free(sky);
    free(alpha_sky);
    free(e1c);
    free(e2c);
    return 0;
}
