/* Plain FP64 CPU oracle for one CCPR time-domain adjoint gradient evaluation.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the benchmark's
 * CPU-baseline leg, never by the product path.  It shares no code with the CUDA library.
 *
 * Everything is written as plain loops over (k, j, i) in double precision, in the order the
 * paper's equations state it; the only parallelism is an OpenMP split of the outer k loop,
 * which does not change any arithmetic.  Readings of the paper where it is silent are listed
 * at the top of each routine.
 *
 * Physical constants: c0 = 299 792 458 m/s, mu0 = 1.25663706212e-6 H/m (CODATA 2018),
 * eps0 = 1/(mu0 c0^2).
 */
#include "fdtd_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const double C0 = 299792458.0;
static const double MU0 = 1.25663706212e-6;
#define EPS0 (1.0 / (MU0 * C0 * C0))
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    double eps_inf[3], sigma[3];
    int np[3];
    cplx* a[3];
    cplx* c[3];
} mat_t;

typedef struct tangent_t tangent_t;

struct oracle_ctx {
    oracle_grid_desc g;
    const tangent_t* tan;     /* non-NULL while update_E advances tangent fields (oracle_tangent) */
    double* freqs;
    double* fw;
    double dt;
    int n[3];
    size_t ncell;
    double* E[3];
    double* H[3];
    double* psiE[3][3]; /* [field component][derivative axis], NULL when equal */
    double* psiH[3][3];
    double* kE[3]; double* bE[3]; double* cE[3];   /* CPML at integer positions  (E updates) */
    double* kH[3]; double* bH[3]; double* cH[3];   /* CPML at half-integer positions (H updates) */
    int have_mat, have_rho, have_fwd, have_adj;
    mat_t bg, m1, m2;
    double gamma;
    int P[3], P1[3];          /* poles per component: m1's first (P1), then m2's */
    cplx* alpha[3];
    cplx* beta[3];
    int wb[6];                /* working box: design box (layout 0), grown by one on +x,+y,+z (layout 1) */
    int sbox[3][6];           /* per component: the voxels whose E_k sample is a design sample */
    size_t soff[4];           /* layout 1: offsets of the components' samples in the density vector */
    int dn[3];                /* working-box extents */
    size_t nd;                /* working-box voxels */
    size_t nvar;              /* design variables */
    double* rho;              /* [nvar] */
    cplx* Q[3];               /* [nd][P[c]] */
    int gn[3];
    size_t ngap;
    cplx* dft[2];             /* forward, adjoint: [F][3][nd] */
    double* src;              /* dipole drive S^{n+1/2}, n = 0..M-1 */
    double* einc;             /* E_inc^n at the first total-field plane */
    double* hinc;             /* H_inc^{n+1/2} half a cell before it */
    double* adjw;             /* adjoint drive [3*ngap][M] */
    double* wave;             /* copy of src_wave, or NULL */
    int inc_ready;            /* einc/hinc built for the current background */
    double F;
    char err[512];
};

static int fail(oracle_ctx* c, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof c->err, fmt, ap);
    va_end(ap);
    return 1;
}

static size_t lin(const oracle_ctx* c, int i, int j, int k)
{
    return ((size_t)k * c->n[1] + j) * c->n[0] + i;
}

/* Field value at (i,j,k); outside the grid it is the periodic image or, behind a PEC wall, 0. */
static double at(const oracle_ctx* c, const double* f, int i, int j, int k)
{
    int idx[3] = {i, j, k};
    for (int a = 0; a < 3; ++a) {
        if (idx[a] < 0 || idx[a] >= c->n[a]) {
            if (c->g.bc[a] == 1)
                idx[a] = (idx[a] % c->n[a] + c->n[a]) % c->n[a];
            else
                return 0.0;
        }
    }
    return f[lin(c, idx[0], idx[1], idx[2])];
}

static int in_box(const int* b, int i, int j, int k)
{
    return i >= b[0] && i < b[1] && j >= b[2] && j < b[3] && k >= b[4] && k < b[5];
}

static int box_empty(const int* b) { return b[1] <= b[0] || b[3] <= b[2] || b[5] <= b[4]; }

/* ---------------------------------------------------------------------------------------------
 * CPML profile (the paper gives only the thickness, 20 cells).  Reading: CFS-CPML with
 * polynomial grading of order m, sigma_max = scale * 0.8 (m+1) / (eta0 dx), kappa graded from 1
 * to kappa_max, a = a_max (1 - d) inside the layer; d is the depth fraction measured from the
 * inner interface (0) to the outer wall (1) at the sample's own (integer or half-integer)
 * position.  psi <- b psi + c dF, derivative replaced by dF/kappa + psi.
 * ------------------------------------------------------------------------------------------- */
static double pml_depth(int lo, int hi, int n, double u)
{
    if (lo > 0 && u < (double)lo) return ((double)lo - u) / (double)lo;
    if (hi > 0 && u > (double)(n - hi)) return (u - (double)(n - hi)) / (double)hi;
    return 0.0;
}

static void pml_coeffs(const oracle_ctx* c, int axis, double u, double* kap, double* b, double* cc)
{
    const oracle_grid_desc* g = &c->g;
    double d = pml_depth(g->cpml[2 * axis], g->cpml[2 * axis + 1], c->n[axis], u);
    double m = g->cpml_m;
    double eta0 = MU0 * C0;
    double smax = g->cpml_sigma_scale * 0.8 * (m + 1.0) / (eta0 * g->dx);
    double sig = d > 0.0 ? smax * pow(d, m) : 0.0;
    double k = d > 0.0 ? 1.0 + (g->cpml_kappa_max - 1.0) * pow(d, m) : 1.0;
    double a = d > 0.0 ? g->cpml_a_max * (1.0 - d) : 0.0;
    *kap = k;
    *b = exp(-(sig / k + a) * c->dt / EPS0);
    *cc = sig > 0.0 ? sig * (*b - 1.0) / (sig * k + k * k * a) : 0.0;
}

static double stretched(double dF, double kap, double b, double cc, double* psi)
{
    *psi = b * (*psi) + cc * dF;
    return dF / kap + *psi;
}

/* ---------------------------------------------------------------------------------------------
 * Source pulse: Gaussian-modulated sine exp(-(t-t0)^2/(2 tau^2)) sin(2 pi f0 (t-t0)); tau from the
 * full width at half maximum of the amplitude spectrum, tau = sqrt(2 ln 2)/(pi fwhm); t0 = 4 tau
 * unless given.  (The configurations give a centre wavelength and a bandwidth only.)
 * ------------------------------------------------------------------------------------------- */
static double src_tau(const oracle_grid_desc* g) { return sqrt(2.0 * log(2.0)) / (M_PI * g->src_fwhm_hz); }
static double src_t0(const oracle_grid_desc* g) { return g->src_t0 > 0.0 ? g->src_t0 : 4.0 * src_tau(g); }

/* Source waveform p(t) (t a multiple of dt/2): the caller's samples if given, else the Gaussian pulse. */
static double pulse_w(const oracle_grid_desc* g, double dt, double t)
{
    if (g->src_wave) {
        long s = lround(2.0 * t / dt);
        return (s >= 0 && s <= 2L * g->n_steps) ? g->src_wave[s] : 0.0;
    }
    double tau = src_tau(g), t0 = src_t0(g);
    double x = t - t0;
    return exp(-x * x / (2.0 * tau * tau)) * sin(2.0 * M_PI * g->src_f0 * x);
}

static void free_mat(mat_t* m)
{
    for (int k = 0; k < 3; ++k) {
        free(m->a[k]);
        free(m->c[k]);
        m->a[k] = m->c[k] = NULL;
        m->np[k] = 0;
    }
}

void oracle_destroy(oracle_ctx* c)
{
    if (!c) return;
    for (int a = 0; a < 3; ++a) {
        free(c->E[a]); free(c->H[a]);
        for (int b = 0; b < 3; ++b) { free(c->psiE[a][b]); free(c->psiH[a][b]); }
        free(c->kE[a]); free(c->bE[a]); free(c->cE[a]);
        free(c->kH[a]); free(c->bH[a]); free(c->cH[a]);
        free(c->alpha[a]); free(c->beta[a]); free(c->Q[a]);
    }
    free_mat(&c->bg); free_mat(&c->m1); free_mat(&c->m2);
    free(c->freqs); free(c->fw); free(c->rho); free(c->wave);
    free(c->dft[0]); free(c->dft[1]);
    free(c->src); free(c->einc); free(c->hinc); free(c->adjw);
    free(c);
}

double oracle_dt(const oracle_ctx* c) { return c ? c->dt : 0.0; }
const char* oracle_last_error(const oracle_ctx* c) { return c ? c->err : "null context"; }

static void* zalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

int oracle_create(const oracle_grid_desc* d, oracle_ctx** out)
{
    if (!d || !out) return 1;
    *out = NULL;
    oracle_ctx* c = (oracle_ctx*)calloc(1, sizeof *c);
    if (!c) return 2;
    c->g = *d;
    c->n[0] = d->nx; c->n[1] = d->ny; c->n[2] = d->nz;
    for (int a = 0; a < 3; ++a) {
        if (c->n[a] < 2) { fail(c, "grid axis %d has %d cells", a, c->n[a]); goto bad; }
        if (d->bc[a] != 0 && d->bc[a] != 1) { fail(c, "bad boundary code"); goto bad; }
        if (d->bc[a] == 1 && (d->cpml[2 * a] || d->cpml[2 * a + 1])) { fail(c, "periodic axis with CPML"); goto bad; }
        if (d->cpml[2 * a] < 0 || d->cpml[2 * a + 1] < 0 || d->cpml[2 * a] + d->cpml[2 * a + 1] > c->n[a]) {
            fail(c, "bad CPML thickness"); goto bad;
        }
    }
    if (!(d->dx > 0.0) || !(d->courant > 0.0) || d->n_steps < 0 || d->n_freq < 0) { fail(c, "bad dx/courant/steps"); goto bad; }
    c->dt = d->courant * d->dx / C0;
    c->ncell = (size_t)d->nx * d->ny * d->nz;
    const int* db = d->design_box;
    const int* gb = d->gap_box;
    if (d->density_layout != 0 && d->density_layout != 1) { fail(c, "bad density layout"); goto bad; }
    memcpy(c->wb, db, sizeof c->wb);
    for (int comp = 0; comp < 3; ++comp) memcpy(c->sbox[comp], db, sizeof c->sbox[comp]);
    if (!box_empty(db)) {
        for (int a = 0; a < 3; ++a)
            if (db[2 * a] < 0 || db[2 * a + 1] > c->n[a]) { fail(c, "design box outside grid"); goto bad; }
        if (d->density_layout == 1) {
            for (int a = 0; a < 3; ++a) {
                c->wb[2 * a + 1] += 1;
                if (c->wb[2 * a + 1] > c->n[a]) { fail(c, "design box + 1 outside grid"); goto bad; }
                for (int comp = 0; comp < 3; ++comp)
                    if (comp != a) c->sbox[comp][2 * a + 1] += 1;
            }
        }
        for (int a = 0; a < 3; ++a) c->dn[a] = c->wb[2 * a + 1] - c->wb[2 * a];
    }
    c->nd = (size_t)c->dn[0] * c->dn[1] * c->dn[2];
    c->nvar = c->nd;
    if (d->density_layout == 1) {
        c->soff[0] = 0;
        for (int comp = 0; comp < 3; ++comp) {
            const int* b = c->sbox[comp];
            c->soff[comp + 1] = c->soff[comp] + (box_empty(db) ? 0 : (size_t)(b[1] - b[0]) * (b[3] - b[2]) * (b[5] - b[4]));
        }
        c->nvar = c->soff[3];
    }
    if (!box_empty(gb)) {
        if (box_empty(db)) { fail(c, "gap without design box"); goto bad; }
        for (int a = 0; a < 3; ++a) {
            if (gb[2 * a] < db[2 * a] || gb[2 * a + 1] > db[2 * a + 1]) { fail(c, "gap box not inside design box"); goto bad; }
            c->gn[a] = gb[2 * a + 1] - gb[2 * a];
        }
    }
    c->ngap = (size_t)c->gn[0] * c->gn[1] * c->gn[2];
    c->freqs = (double*)zalloc((size_t)d->n_freq, sizeof(double));
    c->fw = (double*)zalloc((size_t)d->n_freq, sizeof(double));
    for (int f = 0; f < d->n_freq; ++f) {
        c->freqs[f] = d->freqs_hz[f];
        c->fw[f] = d->freq_weights ? d->freq_weights[f] : 1.0;
    }
    c->g.freqs_hz = c->freqs;
    c->g.freq_weights = c->fw;
    if (d->src_wave) {
        c->wave = (double*)zalloc(2 * (size_t)d->n_steps + 1, sizeof(double));
        memcpy(c->wave, d->src_wave, (2 * (size_t)d->n_steps + 1) * sizeof(double));
    }
    c->g.src_wave = c->wave;
    for (int a = 0; a < 3; ++a) {
        c->E[a] = (double*)zalloc(c->ncell, sizeof(double));
        c->H[a] = (double*)zalloc(c->ncell, sizeof(double));
        for (int b = 0; b < 3; ++b) {
            if (a == b) continue;
            c->psiE[a][b] = (double*)zalloc(c->ncell, sizeof(double));
            c->psiH[a][b] = (double*)zalloc(c->ncell, sizeof(double));
        }
        int na = c->n[a];
        c->kE[a] = (double*)zalloc((size_t)na, sizeof(double));
        c->bE[a] = (double*)zalloc((size_t)na, sizeof(double));
        c->cE[a] = (double*)zalloc((size_t)na, sizeof(double));
        c->kH[a] = (double*)zalloc((size_t)na, sizeof(double));
        c->bH[a] = (double*)zalloc((size_t)na, sizeof(double));
        c->cH[a] = (double*)zalloc((size_t)na, sizeof(double));
        for (int l = 0; l < na; ++l) {
            pml_coeffs(c, a, (double)l, &c->kE[a][l], &c->bE[a][l], &c->cE[a][l]);
            pml_coeffs(c, a, (double)l + 0.5, &c->kH[a][l], &c->bH[a][l], &c->cH[a][l]);
        }
    }
    for (int f = 0; f < 2; ++f) c->dft[f] = (cplx*)zalloc((size_t)d->n_freq * 3 * c->nd, sizeof(cplx));
    c->rho = (double*)zalloc(c->nvar, sizeof(double));
    int M = d->n_steps;
    c->src = (double*)zalloc((size_t)M, sizeof(double));
    c->einc = (double*)zalloc((size_t)M, sizeof(double));
    c->hinc = (double*)zalloc((size_t)M, sizeof(double));
    c->adjw = (double*)zalloc(3 * c->ngap * (size_t)M, sizeof(double));
    if (d->src_kind == 0) {
        for (int a = 0; a < 3; ++a)
            if (d->src_pos[a] < 0 || d->src_pos[a] >= c->n[a]) { fail(c, "dipole outside grid"); goto bad; }
        if (d->src_comp < 0 || d->src_comp > 2) { fail(c, "bad dipole component"); goto bad; }
        /* soft source of amplitude A (V/m per step in vacuum): drive = A (eps0/dt) p(t) */
        for (int n = 0; n < M; ++n) c->src[n] = d->src_amp * (EPS0 / c->dt) * pulse_w(&c->g, c->dt, (n + 0.5) * c->dt);
    } else if (d->src_kind == 1) {
        int i0 = d->src_pos[0];
        if (i0 < d->cpml[0] + 1 || i0 >= c->n[0] - d->cpml[1]) { fail(c, "TF/SF plane inside the CPML"); goto bad; }
    } else {
        fail(c, "bad source kind");
        goto bad;
    }
    *out = c;
    return 0;
bad:
    fprintf(stderr, "oracle_create: %s\n", c->err);
    oracle_destroy(c);
    return 1;
}

static int copy_mat(oracle_ctx* c, mat_t* dst, const oracle_material* m)
{
    free_mat(dst);
    for (int k = 0; k < 3; ++k) {
        dst->eps_inf[k] = m->eps_inf[k];
        dst->sigma[k] = m->sigma[k];
        dst->np[k] = m->n_poles[k];
        if (m->n_poles[k] < 0) return fail(c, "negative pole count");
        dst->a[k] = (cplx*)zalloc((size_t)m->n_poles[k], sizeof(cplx));
        dst->c[k] = (cplx*)zalloc((size_t)m->n_poles[k], sizeof(cplx));
        for (int p = 0; p < m->n_poles[k]; ++p) {
            dst->a[k][p] = m->a_re[k][p] + I * m->a_im[k][p];
            dst->c[k][p] = m->c_re[k][p] + I * m->c_im[k][p];
            /* passive or lossless poles only: Re(a) <= 0, a != 0 (|alpha| <= 1) */
            if (!(m->a_re[k][p] <= 0.0) || (m->a_re[k][p] == 0.0 && m->a_im[k][p] == 0.0))
                return fail(c, "pole with Re(a) > 0 or a = 0");
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------------------------------
 * Pole recursion (ADE of Eq. (Maxwells2)b: dQ/dt = a Q + eps0 c E).  Reading: the paper defers
 * the discretisation to its ref. [material]; here Q is integrated exactly over one step with E
 * held at its trapezoidal mean (E^{n+1}+E^n)/2:
 *     Q^{n+1} = alpha Q^n + beta (E^{n+1} + E^n),  alpha = e^{a dt},  beta = eps0 c (e^{a dt}-1)/(2a).
 * ------------------------------------------------------------------------------------------- */
int oracle_set_materials(oracle_ctx* c, const oracle_material* bg, const oracle_material* m1,
                         const oracle_material* m2, double gamma)
{
    if (!c || !bg || !m1 || !m2) return 1;
    if (copy_mat(c, &c->bg, bg) || copy_mat(c, &c->m1, m1) || copy_mat(c, &c->m2, m2)) return 1;
    for (int k = 0; k < 3; ++k)
        if (c->bg.np[k]) return fail(c, "background material must be non-dispersive");
    c->gamma = gamma;
    c->inc_ready = 0;
    for (int k = 0; k < 3; ++k) {
        free(c->alpha[k]); free(c->beta[k]); free(c->Q[k]);
        c->P1[k] = c->m1.np[k];
        c->P[k] = c->m1.np[k] + c->m2.np[k];
        c->alpha[k] = (cplx*)zalloc((size_t)c->P[k], sizeof(cplx));
        c->beta[k] = (cplx*)zalloc((size_t)c->P[k], sizeof(cplx));
        for (int p = 0; p < c->P[k]; ++p) {
            cplx a = p < c->P1[k] ? c->m1.a[k][p] : c->m2.a[k][p - c->P1[k]];
            cplx cc = p < c->P1[k] ? c->m1.c[k][p] : c->m2.c[k][p - c->P1[k]];
            cplx e = cexp(a * c->dt);
            c->alpha[k][p] = e;
            c->beta[k][p] = EPS0 * cc * (e - 1.0) / (2.0 * a);
        }
        c->Q[k] = (cplx*)zalloc(c->nd * (size_t)(c->P[k] ? c->P[k] : 1), sizeof(cplx));
    }
    c->have_mat = 1;
    c->have_fwd = c->have_adj = 0;
    return 0;
}

int oracle_set_density(oracle_ctx* c, const double* rho, size_t n)
{
    if (!c || (!rho && n)) return 1;
    if (n != c->nvar) return fail(c, "density has %zu values, the design has %zu", n, c->nvar);
    for (size_t v = 0; v < n; ++v)
        if (!(rho[v] >= 0.0 && rho[v] <= 1.0)) return fail(c, "density %zu out of [0,1]", v);
    memcpy(c->rho, rho, n * sizeof(double));
    c->have_rho = 1;
    c->have_fwd = c->have_adj = 0;
    return 0;
}

int oracle_reset(oracle_ctx* c)
{
    for (int a = 0; a < 3; ++a) {
        memset(c->E[a], 0, c->ncell * sizeof(double));
        memset(c->H[a], 0, c->ncell * sizeof(double));
        for (int b = 0; b < 3; ++b) {
            if (c->psiE[a][b]) memset(c->psiE[a][b], 0, c->ncell * sizeof(double));
            if (c->psiH[a][b]) memset(c->psiH[a][b], 0, c->ncell * sizeof(double));
        }
        if (c->Q[a]) memset(c->Q[a], 0, c->nd * (size_t)(c->P[a] ? c->P[a] : 1) * sizeof(cplx));
    }
    return 0;
}

/* ---------------------------------------------------------------------------------------------
 * E update of one sample of a design voxel, centred at n+1/2 (Eq. (Maxwells2)a with the blended
 * model of Eqs. (eps_mixed), (sigma_mixed), (Poles_mixed)):
 *   eps0 eps_inf(rho) (E^{n+1}-E^n)/dt + sigma(rho) (E^{n+1}+E^n)/2
 *       + (2/dt) sum_i kappa_i(rho) sum_p Re{Q_p^{n+1} - Q_p^n} = drive^{n+1/2},
 * drive = (curl H)_k + source, kappa_1 = 1-rho (m1's poles), kappa_2 = rho (m2's poles).
 * Substituting the pole recursion gives E^{n+1}; then each Q_p is advanced.
 * ------------------------------------------------------------------------------------------- */
static double design_sample_update(const oracle_ctx* c, int comp, double rho, cplx* Q, double e_old, double drive)
{
    const double dt = c->dt;
    double kap1 = 1.0 - rho, kap2 = rho;
    double eps = kap1 * c->m1.eps_inf[comp] + kap2 * c->m2.eps_inf[comp];
    double sig = kap1 * c->m1.sigma[comp] + kap2 * c->m2.sigma[comp] + rho * (1.0 - rho) * c->gamma;
    double sum_re_beta = 0.0, sum_re_aq = 0.0;
    for (int p = 0; p < c->P[comp]; ++p) {
        double kp = p < c->P1[comp] ? kap1 : kap2;
        sum_re_beta += kp * creal(c->beta[comp][p]);
        sum_re_aq += kp * creal((c->alpha[comp][p] - 1.0) * Q[p]);
    }
    double D = EPS0 * eps / dt + sig / 2.0 + 2.0 * sum_re_beta / dt;
    double N = EPS0 * eps / dt - sig / 2.0 - 2.0 * sum_re_beta / dt;
    double e_new = (N * e_old + drive - 2.0 * sum_re_aq / dt) / D;
    for (int p = 0; p < c->P[comp]; ++p)
        Q[p] = c->alpha[comp][p] * Q[p] + c->beta[comp][p] * (e_new + e_old);
    return e_new;
}

static double background_sample_update(const oracle_ctx* c, int comp, double e_old, double drive)
{
    const double dt = c->dt;
    double eps = c->bg.eps_inf[comp], sig = c->bg.sigma[comp];
    double D = EPS0 * eps / dt + sig / 2.0;
    double N = EPS0 * eps / dt - sig / 2.0;
    return (N * e_old + drive) / D;
}

/* Tangent-linear mode (oracle_tangent): derivative fields dE, dH, dpsi, dQ of the forward run in a
 * density direction drho, advanced by the same discrete scheme differentiated by hand.  While
 * update_E runs on the swapped-in tangent arrays, `tan` holds the primal E^n, E^{n+1} and Q^n. */
struct tangent_t {
    const double* E0[3];    /* primal E^n (copy) */
    const double* E1[3];    /* primal E^{n+1} */
    const cplx* Q0[3];      /* primal Q^n (copy) */
    const double* drho;     /* direction over the design variables */
};

/* dE^{n+1} of one sample.  Background samples: the same linear update on (dE^n, d curl).  Design
 * samples: differentiating D(rho) E^{n+1} = N(rho) E^n + drive - (2/dt) sum_p kappa_p(rho) Re{(alpha_p-1) Q_p^n}
 *   D dE^{n+1} = N dE^n + d drive - (2/dt) sum_p kappa_p Re{(alpha_p-1) dQ_p^n}
 *                + drho [N' E^n - (2/dt) sum_p kappa_p' Re{(alpha_p-1) Q_p^n} - D' E^{n+1}],
 * with kappa' = -1 for m1's poles and +1 for m2's and D', N' the rho-derivatives of D, N (eps_inf, sigma
 * with the rho(1-rho) gamma term, and sum kappa Re beta); then dQ_p <- alpha_p dQ_p + beta_p (dE^{n+1} + dE^n). */
static double tangent_sample_update(const oracle_ctx* c, int comp, int i, int j, int k, size_t p, int cls, size_t dv,
                                    double de_old, double ddrive);

int oracle_sample_response(oracle_ctx* c, int comp, double rho, int n, const double* curl, double* e_out)
{
    if (!c || !c->have_mat || comp < 0 || comp > 2) return 1;
    cplx* Q = (cplx*)zalloc((size_t)(c->P[comp] ? c->P[comp] : 1), sizeof(cplx));
    double e = 0.0;
    for (int s = 0; s < n; ++s) {
        e = design_sample_update(c, comp, rho, Q, e, curl[s]);
        e_out[s] = e;
    }
    free(Q);
    return 0;
}

/* E sample fixed at zero by a PEC wall: the components tangential to the wall at index 0. */
static int pec_fixed(const oracle_ctx* c, int comp, const int* ijk)
{
    for (int a = 0; a < 3; ++a)
        if (a != comp && c->g.bc[a] == 0 && ijk[a] == 0) return 1;
    return 0;
}

/* class of a voxel: 0 background, 1 in the working box (design state kept), 2 gap (fixed
 * background inside the box) */
static int voxel_class(const oracle_ctx* c, int i, int j, int k)
{
    if (c->nd == 0 || !in_box(c->wb, i, j, k)) return 0;
    if (c->ngap && in_box(c->g.gap_box, i, j, k)) return 2;
    return 1;
}

/* E_comp of voxel (i,j,k) is a design (blended) sample */
static int design_sample(const oracle_ctx* c, int comp, int i, int j, int k)
{
    return voxel_class(c, i, j, k) == 1 && in_box(c->sbox[comp], i, j, k);
}

static size_t design_index(const oracle_ctx* c, int i, int j, int k)
{
    const int* b = c->wb;
    return ((size_t)(k - b[4]) * c->dn[1] + (j - b[2])) * c->dn[0] + (i - b[0]);
}

/* position of the density of design sample E_comp(i,j,k) in the density vector */
static size_t rho_index(const oracle_ctx* c, int comp, int i, int j, int k)
{
    if (c->g.density_layout != 1) return design_index(c, i, j, k);
    const int* b = c->sbox[comp];
    return c->soff[comp] + ((size_t)(k - b[4]) * (b[3] - b[2]) + (j - b[2])) * (b[1] - b[0]) + (i - b[0]);
}

static size_t gap_index(const oracle_ctx* c, int i, int j, int k)
{
    const int* b = c->g.gap_box;
    return ((size_t)(k - b[4]) * c->gn[1] + (j - b[2])) * c->gn[0] + (i - b[0]);
}

static double tangent_sample_update(const oracle_ctx* c, int comp, int i, int j, int k, size_t p, int cls, size_t dv,
                                    double de_old, double ddrive)
{
    const tangent_t* t = c->tan;
    if (!(cls == 1 && design_sample(c, comp, i, j, k))) return background_sample_update(c, comp, de_old, ddrive);
    const double dt = c->dt;
    const size_t r = rho_index(c, comp, i, j, k);
    const double rho = c->rho[r], drho = t->drho[r];
    const int P = c->P[comp];
    cplx* dQ = &c->Q[comp][dv * (size_t)P];              /* tangent pole currents (swapped in) */
    const cplx* Q0 = &t->Q0[comp][dv * (size_t)P];
    const double e0 = t->E0[comp][p], e1 = t->E1[comp][p];
    const double kap1 = 1.0 - rho, kap2 = rho;
    const double eps = kap1 * c->m1.eps_inf[comp] + kap2 * c->m2.eps_inf[comp];
    const double sig = kap1 * c->m1.sigma[comp] + kap2 * c->m2.sigma[comp] + rho * (1.0 - rho) * c->gamma;
    const double eps_r = c->m2.eps_inf[comp] - c->m1.eps_inf[comp];
    const double sig_r = c->m2.sigma[comp] - c->m1.sigma[comp] + (1.0 - 2.0 * rho) * c->gamma;
    double srb = 0.0, srb_r = 0.0, saq_d = 0.0, saq_r = 0.0;
    for (int q = 0; q < P; ++q) {
        const double kq = q < c->P1[comp] ? kap1 : kap2, kq_r = q < c->P1[comp] ? -1.0 : 1.0;
        srb += kq * creal(c->beta[comp][q]);
        srb_r += kq_r * creal(c->beta[comp][q]);
        saq_d += kq * creal((c->alpha[comp][q] - 1.0) * dQ[q]);
        saq_r += kq_r * creal((c->alpha[comp][q] - 1.0) * Q0[q]);
    }
    const double D = EPS0 * eps / dt + sig / 2.0 + 2.0 * srb / dt;
    const double N = EPS0 * eps / dt - sig / 2.0 - 2.0 * srb / dt;
    const double D_r = EPS0 * eps_r / dt + sig_r / 2.0 + 2.0 * srb_r / dt;
    const double N_r = EPS0 * eps_r / dt - sig_r / 2.0 - 2.0 * srb_r / dt;
    const double de_new = (N * de_old + ddrive - 2.0 * saq_d / dt + drho * (N_r * e0 - 2.0 * saq_r / dt - D_r * e1)) / D;
    for (int q = 0; q < P; ++q) dQ[q] = c->alpha[comp][q] * dQ[q] + c->beta[comp][q] * (de_new + de_old);
    return de_new;
}

/* H^{n+1/2} = H^{n-1/2} - (dt/mu0) curl E^n  (Eq. (Maxwells2)c), CPML-stretched derivatives. */
static void update_H(oracle_ctx* c, int n, int mode)
{
    const int nx = c->n[0], ny = c->n[1], nz = c->n[2];
    const double ch = c->dt / MU0, idx = 1.0 / c->g.dx;
    const int tfsf = (mode == 1 && c->g.src_kind == 1);
    const int i0 = c->g.src_pos[0];
    double *Ex = c->E[0], *Ey = c->E[1], *Ez = c->E[2];
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t p = lin(c, i, j, k);
                /* H_x at (i, j+1/2, k+1/2): (curl E)_x = dEz/dy - dEy/dz */
                double dEz_dy = (at(c, Ez, i, j + 1, k) - Ez[p]) * idx;
                double dEy_dz = (at(c, Ey, i, j, k + 1) - Ey[p]) * idx;
                double cx = stretched(dEz_dy, c->kH[1][j], c->bH[1][j], c->cH[1][j], &c->psiH[0][1][p])
                          - stretched(dEy_dz, c->kH[2][k], c->bH[2][k], c->cH[2][k], &c->psiH[0][2][p]);
                c->H[0][p] -= ch * cx;
                /* H_y at (i+1/2, j, k+1/2): (curl E)_y = dEx/dz - dEz/dx */
                double dEx_dz = (at(c, Ex, i, j, k + 1) - Ex[p]) * idx;
                double dEz_dx = (at(c, Ez, i + 1, j, k) - Ez[p]) * idx;
                if (tfsf && i == i0 - 1) dEz_dx -= c->einc[n] * idx; /* H_y here is scattered field */
                double cy = stretched(dEx_dz, c->kH[2][k], c->bH[2][k], c->cH[2][k], &c->psiH[1][2][p])
                          - stretched(dEz_dx, c->kH[0][i], c->bH[0][i], c->cH[0][i], &c->psiH[1][0][p]);
                c->H[1][p] -= ch * cy;
                /* H_z at (i+1/2, j+1/2, k): (curl E)_z = dEy/dx - dEx/dy */
                double dEy_dx = (at(c, Ey, i + 1, j, k) - Ey[p]) * idx;
                double dEx_dy = (at(c, Ex, i, j + 1, k) - Ex[p]) * idx;
                double cz = stretched(dEy_dx, c->kH[0][i], c->bH[0][i], c->cH[0][i], &c->psiH[2][0][p])
                          - stretched(dEx_dy, c->kH[1][j], c->bH[1][j], c->cH[1][j], &c->psiH[2][1][p]);
                c->H[2][p] -= ch * cz;
            }
}

static double point_drive(const oracle_ctx* c, int comp, int i, int j, int k, int n, int mode, int cls)
{
    if (mode == 1 && c->g.src_kind == 0) {
        if (comp == c->g.src_comp && i == c->g.src_pos[0] && j == c->g.src_pos[1] && k == c->g.src_pos[2])
            return c->src[n];
    } else if (mode == 2 && cls == 2) {
        size_t s = (size_t)comp * c->ngap + gap_index(c, i, j, k);
        return c->adjw[s * (size_t)c->g.n_steps + n];
    }
    return 0.0;
}

/* E^{n+1} from E^n, curl H^{n+1/2} (CPML-stretched), the source and the pole currents. */
static void update_E(oracle_ctx* c, int n, int mode)
{
    const int nx = c->n[0], ny = c->n[1], nz = c->n[2];
    const double idx = 1.0 / c->g.dx;
    const int tfsf = (mode == 1 && c->g.src_kind == 1);
    const int i0 = c->g.src_pos[0];
    double *Hx = c->H[0], *Hy = c->H[1], *Hz = c->H[2];
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t p = lin(c, i, j, k);
                int ijk[3] = {i, j, k};
                int cls = voxel_class(c, i, j, k);
                size_t dv = cls ? design_index(c, i, j, k) : 0;
                for (int comp = 0; comp < 3; ++comp) {
                    if (pec_fixed(c, comp, ijk)) continue;
                    double curl;
                    if (comp == 0) { /* E_x at (i+1/2, j, k): dHz/dy - dHy/dz */
                        double dHz_dy = (Hz[p] - at(c, Hz, i, j - 1, k)) * idx;
                        double dHy_dz = (Hy[p] - at(c, Hy, i, j, k - 1)) * idx;
                        curl = stretched(dHz_dy, c->kE[1][j], c->bE[1][j], c->cE[1][j], &c->psiE[0][1][p])
                             - stretched(dHy_dz, c->kE[2][k], c->bE[2][k], c->cE[2][k], &c->psiE[0][2][p]);
                    } else if (comp == 1) { /* E_y at (i, j+1/2, k): dHx/dz - dHz/dx */
                        double dHx_dz = (Hx[p] - at(c, Hx, i, j, k - 1)) * idx;
                        double dHz_dx = (Hz[p] - at(c, Hz, i - 1, j, k)) * idx;
                        curl = stretched(dHx_dz, c->kE[2][k], c->bE[2][k], c->cE[2][k], &c->psiE[1][2][p])
                             - stretched(dHz_dx, c->kE[0][i], c->bE[0][i], c->cE[0][i], &c->psiE[1][0][p]);
                    } else { /* E_z at (i, j, k+1/2): dHy/dx - dHx/dy */
                        double dHy_dx = (Hy[p] - at(c, Hy, i - 1, j, k)) * idx;
                        if (tfsf && i == i0) dHy_dx -= c->hinc[n] * idx; /* H_y(i0-1/2) is scattered field */
                        double dHx_dy = (Hx[p] - at(c, Hx, i, j - 1, k)) * idx;
                        curl = stretched(dHy_dx, c->kE[0][i], c->bE[0][i], c->cE[0][i], &c->psiE[2][0][p])
                             - stretched(dHx_dy, c->kE[1][j], c->bE[1][j], c->cE[1][j], &c->psiE[2][1][p]);
                    }
                    double drive = curl + point_drive(c, comp, i, j, k, n, mode, cls);
                    double* e = &c->E[comp][p];
                    if (c->tan)
                        *e = tangent_sample_update(c, comp, i, j, k, p, cls, dv, *e, drive);
                    else if (cls == 1 && design_sample(c, comp, i, j, k))
                        *e = design_sample_update(c, comp, c->rho[rho_index(c, comp, i, j, k)],
                                                  &c->Q[comp][dv * (size_t)c->P[comp]], *e, drive);
                    else
                        *e = background_sample_update(c, comp, *e, drive);
                }
            }
}

/* ---------------------------------------------------------------------------------------------
 * Incident plane wave for the one-sided TF/SF plane (reading: the paper injects a plane wave but
 * gives no injection scheme).  A 1-D Yee line along x with the same dx, dt and the background's
 * z-component material carries E_z/H_y from a hard source at its first node; node `off` maps onto
 * the first total-field plane x = i0 dx and H node off-1 onto x = (i0-1/2) dx.  The line is long
 * enough that its far-end reflection never returns within n_steps.
 * ------------------------------------------------------------------------------------------- */
static void build_incident(oracle_ctx* c)
{
    const oracle_grid_desc* g = &c->g;
    if (c->inc_ready) return;
    c->inc_ready = 1;
    const int M = g->n_steps, off = 2;
    const int L = off + (int)ceil(0.6 * M) + 16;
    double* e1 = (double*)zalloc((size_t)L, sizeof(double));
    double* h1 = (double*)zalloc((size_t)L, sizeof(double));
    const double dt = c->dt, dx = g->dx;
    double eps = c->bg.eps_inf[2], sig = c->bg.sigma[2];
    double D = EPS0 * eps / dt + sig / 2.0, N = EPS0 * eps / dt - sig / 2.0;
    e1[0] = g->src_amp * pulse_w(g, dt, 0.0);
    for (int n = 0; n < M; ++n) {
        c->einc[n] = e1[off];
        for (int m = 0; m < L; ++m) {
            double e_next = m + 1 < L ? e1[m + 1] : 0.0;
            h1[m] += dt / (MU0 * dx) * (e_next - e1[m]);
        }
        c->hinc[n] = h1[off - 1];
        for (int m = 1; m < L; ++m) e1[m] = (N * e1[m] + (h1[m] - h1[m - 1]) / dx) / D;
        e1[0] = g->src_amp * pulse_w(g, dt, (n + 1) * dt);
    }
    free(e1);
    free(h1);
}

static void step_once(oracle_ctx* c, int n, int mode)
{
    update_H(c, n, mode);
    update_E(c, n, mode);
}

int oracle_step(oracle_ctx* c, int n_first, int n_count, int source_mode)
{
    if (!c || !c->have_mat) return 1;
    if (c->nd && !c->have_rho) return fail(c, "density not set");
    if (source_mode && (n_first < 0 || n_first + n_count > c->g.n_steps)) return fail(c, "source table range");
    if (source_mode == 1 && c->g.src_kind == 1 && n_first == 0) c->inc_ready = 0;
    if (source_mode == 1 && c->g.src_kind == 1) build_incident(c);
    for (int s = 0; s < n_count; ++s) step_once(c, n_first + s, source_mode);
    return 0;
}

/* Running DFT (frequency-domain objective; e^{j w t} convention so the forward transform uses
 * e^{-j w t}):  Ehat_s(w) = sum_{n=1..M} E_s^n e^{-j w n dt}.  Reading: the paper stores full
 * histories; this transform over all steps is its running-sum equivalent (no dt factor). */
static void accumulate_dft(oracle_ctx* c, cplx* dft, int nt)
{
    const int* b = c->wb;
    for (int f = 0; f < c->g.n_freq; ++f) {
        cplx ph = cexp(-I * 2.0 * M_PI * c->freqs[f] * (double)nt * c->dt);
        for (int comp = 0; comp < 3; ++comp) {
            cplx* d = dft + ((size_t)f * 3 + comp) * c->nd;
            for (int k = b[4]; k < b[5]; ++k)
                for (int j = b[2]; j < b[3]; ++j)
                    for (int i = b[0]; i < b[1]; ++i)
                        d[design_index(c, i, j, k)] += c->E[comp][lin(c, i, j, k)] * ph;
        }
    }
}

static int run(oracle_ctx* c, int mode)
{
    if (!c->have_mat) return fail(c, "materials not set");
    if (c->nd && !c->have_rho) return fail(c, "density not set");
    oracle_reset(c);
    cplx* dft = c->dft[mode == 2 ? 1 : 0];
    memset(dft, 0, (size_t)c->g.n_freq * 3 * c->nd * sizeof(cplx));
    if (mode == 1 && c->g.src_kind == 1) build_incident(c);
    for (int n = 0; n < c->g.n_steps; ++n) {
        step_once(c, n, mode);
        accumulate_dft(c, dft, n + 1);
    }
    return 0;
}

/* Objective: F = sum_f w_f sum_{s in gap samples} |Ehat_s(w_f)|^2, all three owned components of
 * every gap voxel.  Frequency-domain form of Eq. (Objective_analyitically_enhancement). */
int oracle_forward(oracle_ctx* c, double* F_out, double* gap_dft_out)
{
    if (!c) return 1;
    if (run(c, 1)) return 1;
    const int* gb = c->g.gap_box;
    double F = 0.0;
    for (int f = 0; f < c->g.n_freq; ++f)
        for (int comp = 0; comp < 3; ++comp) {
            const cplx* d = c->dft[0] + ((size_t)f * 3 + comp) * c->nd;
            if (!c->ngap) continue;
            for (int k = gb[4]; k < gb[5]; ++k)
                for (int j = gb[2]; j < gb[3]; ++j)
                    for (int i = gb[0]; i < gb[1]; ++i) {
                        cplx v = d[design_index(c, i, j, k)];
                        F += c->fw[f] * (creal(v) * creal(v) + cimag(v) * cimag(v));
                        if (gap_dft_out) {
                            size_t s = ((size_t)f * 3 + comp) * c->ngap + gap_index(c, i, j, k);
                            gap_dft_out[2 * s] = creal(v);
                            gap_dft_out[2 * s + 1] = cimag(v);
                        }
                    }
        }
    c->F = F;
    if (F_out) *F_out = F;
    c->have_fwd = 1;
    c->have_adj = 0;
    return 0;
}

/* Swap the field, psi and pole-current arrays with the tangent ones. */
static void swap_tangent(oracle_ctx* c, double* tE[3], double* tH[3], double* tpE[3][3], double* tpH[3][3], cplx* tQ[3])
{
    for (int a = 0; a < 3; ++a) {
        double* x = c->E[a]; c->E[a] = tE[a]; tE[a] = x;
        x = c->H[a]; c->H[a] = tH[a]; tH[a] = x;
        for (int b = 0; b < 3; ++b) {
            x = c->psiE[a][b]; c->psiE[a][b] = tpE[a][b]; tpE[a][b] = x;
            x = c->psiH[a][b]; c->psiH[a][b] = tpH[a][b]; tpH[a][b] = x;
        }
        cplx* q = c->Q[a]; c->Q[a] = tQ[a]; tQ[a] = q;
    }
}

/* Forward run with its tangent-linear run in the density direction drho (n = design variables):
 * F and dF = d/de F(rho + e drho) at e = 0, the exact derivative of the discrete objective (the
 * forward-mode counterpart of the adjoint gradient; a check of it free of finite-difference error). */
int oracle_tangent(oracle_ctx* c, const double* drho, size_t n, double* F_out, double* dF_out, double* Ftd_out,
                   double* dFtd_out)
{
    if (!c || !drho) return 1;
    if (!c->have_mat) return fail(c, "materials not set");
    if (c->nd && !c->have_rho) return fail(c, "density not set");
    if (n != c->nvar) return fail(c, "direction has %zu values, the design has %zu", n, c->nvar);
    const int M = c->g.n_steps;
    double* tE[3]; double* tH[3]; double* tpE[3][3]; double* tpH[3][3]; cplx* tQ[3];
    double* E0[3]; cplx* Q0[3];
    for (int a = 0; a < 3; ++a) {
        tE[a] = (double*)zalloc(c->ncell, sizeof(double));
        tH[a] = (double*)zalloc(c->ncell, sizeof(double));
        E0[a] = (double*)zalloc(c->ncell, sizeof(double));
        const size_t nq = c->nd * (size_t)(c->P[a] ? c->P[a] : 1);
        tQ[a] = (cplx*)zalloc(nq, sizeof(cplx));
        Q0[a] = (cplx*)zalloc(nq, sizeof(cplx));
        for (int b = 0; b < 3; ++b) {
            tpE[a][b] = c->psiE[a][b] ? (double*)zalloc(c->ncell, sizeof(double)) : NULL;
            tpH[a][b] = c->psiH[a][b] ? (double*)zalloc(c->ncell, sizeof(double)) : NULL;
        }
    }
    cplx* tdft = (cplx*)zalloc((size_t)c->g.n_freq * 3 * c->nd, sizeof(cplx));
    tangent_t t;
    double std_ = 0.0, dstd = 0.0;   /* time-domain gap energy sum and its tangent */
    const int* gbx = c->g.gap_box;
    oracle_reset(c);
    memset(c->dft[0], 0, (size_t)c->g.n_freq * 3 * c->nd * sizeof(cplx));
    if (c->g.src_kind == 1) { c->inc_ready = 0; build_incident(c); }
    for (int s = 0; s < M; ++s) {
        update_H(c, s, 1);
        swap_tangent(c, tE, tH, tpE, tpH, tQ);
        update_H(c, s, 0);                               /* linear, no source */
        swap_tangent(c, tE, tH, tpE, tpH, tQ);
        for (int a = 0; a < 3; ++a) {
            memcpy(E0[a], c->E[a], c->ncell * sizeof(double));
            memcpy(Q0[a], c->Q[a], c->nd * (size_t)(c->P[a] ? c->P[a] : 1) * sizeof(cplx));
        }
        update_E(c, s, 1);
        for (int a = 0; a < 3; ++a) { t.E0[a] = E0[a]; t.E1[a] = c->E[a]; t.Q0[a] = Q0[a]; }
        t.drho = drho;
        swap_tangent(c, tE, tH, tpE, tpH, tQ);
        c->tan = &t;
        update_E(c, s, 0);
        c->tan = NULL;
        accumulate_dft(c, tdft, s + 1);
        swap_tangent(c, tE, tH, tpE, tpH, tQ);
        accumulate_dft(c, c->dft[0], s + 1);
        for (int comp = 0; comp < 3 && c->ngap; ++comp)
            for (int k = gbx[4]; k < gbx[5]; ++k)
                for (int j = gbx[2]; j < gbx[3]; ++j)
                    for (int i = gbx[0]; i < gbx[1]; ++i) {
                        const size_t p = lin(c, i, j, k);
                        std_ += c->E[comp][p] * c->E[comp][p];
                        dstd += 2.0 * c->E[comp][p] * tE[comp][p];
                    }
    }
    const int* gb = c->g.gap_box;
    double F = 0.0, dF = 0.0;
    for (int f = 0; f < c->g.n_freq && c->ngap; ++f)
        for (int comp = 0; comp < 3; ++comp) {
            const size_t o = ((size_t)f * 3 + comp) * c->nd;
            for (int k = gb[4]; k < gb[5]; ++k)
                for (int j = gb[2]; j < gb[3]; ++j)
                    for (int i = gb[0]; i < gb[1]; ++i) {
                        const size_t v = design_index(c, i, j, k);
                        const cplx e = c->dft[0][o + v], de = tdft[o + v];
                        F += c->fw[f] * (creal(e) * creal(e) + cimag(e) * cimag(e));
                        dF += c->fw[f] * 2.0 * (creal(e) * creal(de) + cimag(e) * cimag(de));
                    }
        }
    for (int a = 0; a < 3; ++a) {
        free(tE[a]); free(tH[a]); free(E0[a]); free(tQ[a]); free(Q0[a]);
        for (int b = 0; b < 3; ++b) { free(tpE[a][b]); free(tpH[a][b]); }
    }
    free(tdft);
    c->have_fwd = 0;
    c->have_adj = 0;
    if (F_out) *F_out = F;
    if (dF_out) *dF_out = dF;
    const double dV = c->g.dx * c->g.dx * c->g.dx;   /* the paper-mode objective's scale */
    if (Ftd_out) *Ftd_out = 0.5 * EPS0 * dV * c->dt * std_;
    if (dFtd_out) *dFtd_out = 0.5 * EPS0 * dV * c->dt * dstd;
    return 0;
}

/* Dense real solve with partial pivoting (A is n x n, row-major; b overwritten by x). */
static int solve_dense(int n, double* A, double* b)
{
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(A[r * n + col]) > fabs(A[piv * n + col])) piv = r;
        if (A[piv * n + col] == 0.0) return 1;
        if (piv != col) {
            for (int q = 0; q < n; ++q) { double t = A[col * n + q]; A[col * n + q] = A[piv * n + q]; A[piv * n + q] = t; }
            double t = b[col]; b[col] = b[piv]; b[piv] = t;
        }
        for (int r = col + 1; r < n; ++r) {
            double f = A[r * n + col] / A[col * n + col];
            for (int q = col; q < n; ++q) A[r * n + q] -= f * A[col * n + q];
            b[r] -= f * b[col];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int q = r + 1; q < n; ++q) s -= A[r * n + q] * b[q];
        b[r] = s / A[r * n + r];
    }
    return 0;
}

/* Adjoint basis pulse q = 2f + s: exp(-(t-t0a)^2/(2 tau_a^2)) x {cos, sin}(w_f (t - t0a)). */
static double adj_basis(const oracle_ctx* c, int q, double t)
{
    double tau = c->g.adj_tau > 0.0 ? c->g.adj_tau : src_tau(&c->g);
    double t0 = 4.0 * tau;
    double x = t - t0;
    double w = 2.0 * M_PI * c->freqs[q / 2];
    double env = exp(-x * x / (2.0 * tau * tau));
    return (q % 2 == 0) ? env * cos(w * x) : env * sin(w * x);
}

/* ---------------------------------------------------------------------------------------------
 * Adjoint run.  The adjoint source is the time-reversed objective derivative (Sec. "Time-domain
 * adjoint formulation", SI Eq. (AdjointSystem)a).  For the DFT objective its spectrum at each w_f
 * must be w_f-weight x conj(Ehat_g(w_f)) at every gap sample g (time reversal = conjugation for
 * the e^{j w t} transform); the discrete Yee/CPML/ADE operator is reciprocal, so the same forward
 * solver yields the adjoint field.  Reading for several frequencies in one run: each gap sample
 * is driven by sum_q r_{g,q} b_q((n+1/2)dt) over 2F real basis pulses, with the real r_g solving
 *     sum_q r_{g,q} sum_{n=0}^{M-1} b_q((n+1/2) dt) e^{-j w_f n dt} = w_f conj(Ehat_g(w_f))
 * (real and imaginary parts: a 2F x 2F real system).
 * ------------------------------------------------------------------------------------------- */
int oracle_adjoint(oracle_ctx* c)
{
    if (!c || !c->have_fwd) return c ? fail(c, "adjoint before forward") : 1;
    if (!c->ngap) return fail(c, "adjoint needs a gap");
    const int F = c->g.n_freq, nb = 2 * F, M = c->g.n_steps;
    double* A0 = (double*)zalloc((size_t)nb * nb, sizeof(double));
    double* A = (double*)zalloc((size_t)nb * nb, sizeof(double));
    double* r = (double*)zalloc((size_t)nb, sizeof(double));
    for (int f = 0; f < F; ++f)
        for (int q = 0; q < nb; ++q) {
            cplx s = 0.0;
            for (int n = 0; n < M; ++n)
                s += adj_basis(c, q, (n + 0.5) * c->dt) * cexp(-I * 2.0 * M_PI * c->freqs[f] * (double)n * c->dt);
            A0[(2 * f) * nb + q] = creal(s);
            A0[(2 * f + 1) * nb + q] = cimag(s);
        }
    const int* gb = c->g.gap_box;
    for (int comp = 0; comp < 3; ++comp)
        for (int k = gb[4]; k < gb[5]; ++k)
            for (int j = gb[2]; j < gb[3]; ++j)
                for (int i = gb[0]; i < gb[1]; ++i) {
                    size_t gs = (size_t)comp * c->ngap + gap_index(c, i, j, k);
                    for (int f = 0; f < F; ++f) {
                        cplx e = c->dft[0][((size_t)f * 3 + comp) * c->nd + design_index(c, i, j, k)];
                        cplx t = c->fw[f] * conj(e);
                        r[2 * f] = creal(t);
                        r[2 * f + 1] = cimag(t);
                    }
                    memcpy(A, A0, (size_t)nb * nb * sizeof(double));
                    if (solve_dense(nb, A, r)) { free(A0); free(A); free(r); return fail(c, "singular adjoint basis"); }
                    for (int n = 0; n < M; ++n) {
                        double s = 0.0;
                        for (int q = 0; q < nb; ++q) s += r[q] * adj_basis(c, q, (n + 0.5) * c->dt);
                        c->adjw[gs * (size_t)M + n] = s;
                    }
                }
    free(A0);
    free(A);
    free(r);
    if (run(c, 2)) return 1;
    c->have_adj = 1;
    return 0;
}

/* ---------------------------------------------------------------------------------------------
 * Paper mode (see the header): the time-domain energy objective and Eq. (Gradient_FDTD) with
 * stored histories.  Histories cover every owned sample of the design box, n = 0..M.
 * ------------------------------------------------------------------------------------------- */
static double gap_energy(const oracle_ctx* c)
{
    const int* gb = c->g.gap_box;
    double s = 0.0;
    for (int comp = 0; comp < 3; ++comp)
        for (int k = gb[4]; k < gb[5]; ++k)
            for (int j = gb[2]; j < gb[3]; ++j)
                for (int i = gb[0]; i < gb[1]; ++i) {
                    double e = c->E[comp][lin(c, i, j, k)];
                    s += e * e;
                }
    return s;
}

static void record_E(const oracle_ctx* c, double* hist, int n, int M)
{
    const int* b = c->g.design_box;
    for (int comp = 0; comp < 3; ++comp)
        for (int k = b[4]; k < b[5]; ++k)
            for (int j = b[2]; j < b[3]; ++j)
                for (int i = b[0]; i < b[1]; ++i) {
                    size_t s = (size_t)comp * c->nd + design_index(c, i, j, k);
                    hist[s * (size_t)(M + 1) + n] = c->E[comp][lin(c, i, j, k)];
                }
}

/* Q histories: [comp][design voxel][pole][n] */
static void record_Q(const oracle_ctx* c, cplx* qh[3], int n, int M)
{
    for (int comp = 0; comp < 3; ++comp)
        for (size_t v = 0; v < c->nd; ++v)
            for (int p = 0; p < c->P[comp]; ++p)
                qh[comp][(v * (size_t)c->P[comp] + p) * (size_t)(M + 1) + n] = c->Q[comp][v * (size_t)c->P[comp] + p];
}

static int paper_forward(oracle_ctx* c, double* F_out, double* eh, cplx* qh[3])
{
    if (!c->have_mat) return fail(c, "materials not set");
    if (c->nd && !c->have_rho) return fail(c, "density not set");
    if (!c->ngap) return fail(c, "paper mode needs a gap");
    if (c->g.density_layout != 0) return fail(c, "paper mode takes one density per voxel");
    const int M = c->g.n_steps;
    oracle_reset(c);
    if (c->g.src_kind == 1) {
        c->inc_ready = 0;
        build_incident(c);
    }
    if (eh) record_E(c, eh, 0, M);
    if (qh[0] || qh[1] || qh[2]) record_Q(c, qh, 0, M);
    double s = 0.0;
    for (int n = 0; n < M; ++n) {
        step_once(c, n, 1);
        s += gap_energy(c);
        if (eh) record_E(c, eh, n + 1, M);
        if (qh[0] || qh[1] || qh[2]) record_Q(c, qh, n + 1, M);
    }
    const double dV = c->g.dx * c->g.dx * c->g.dx;
    *F_out = 0.5 * EPS0 * dV * c->dt * s;
    return 0;
}

int oracle_paper_objective(oracle_ctx* c, double* F_out)
{
    if (!c || !F_out) return 1;
    cplx* none[3] = {NULL, NULL, NULL};
    return paper_forward(c, F_out, NULL, none);
}

int oracle_paper_gradient(oracle_ctx* c, int align, double* F_out, double* grad, size_t n)
{
    if (!c || !grad) return 1;
    if (n != c->nd) return fail(c, "gradient size %zu != %zu design voxels", n, c->nd);
    const int M = c->g.n_steps;
    const size_t ns = 3 * c->nd, L = (size_t)M + 1;
    double* eh = (double*)zalloc(ns * L, sizeof(double));     /* forward E^n */
    double* ah = (double*)zalloc(ns * L, sizeof(double));     /* adjoint Etilde^m */
    cplx* qh[3];
    for (int comp = 0; comp < 3; ++comp) qh[comp] = (cplx*)zalloc(c->nd * (size_t)(c->P[comp] ? c->P[comp] : 1) * L, sizeof(cplx));
    double F = 0.0;
    int rc = paper_forward(c, &F, eh, qh);
    if (!rc) {
        /* adjoint drive at every gap sample: the time-reversed functional derivative eps0 E */
        const int* gb = c->g.gap_box;
        const int delay = align & 1;
        for (int comp = 0; comp < 3; ++comp)
            for (int k = gb[4]; k < gb[5]; ++k)
                for (int j = gb[2]; j < gb[3]; ++j)
                    for (int i = gb[0]; i < gb[1]; ++i) {
                        size_t gs = (size_t)comp * c->ngap + gap_index(c, i, j, k);
                        size_t ds = (size_t)comp * c->nd + design_index(c, i, j, k);
                        for (int m = 0; m < M; ++m) {
                            int nf = M - m - delay;
                            c->adjw[gs * (size_t)M + m] = nf >= 0 ? EPS0 * eh[ds * L + nf] : 0.0;
                        }
                    }
        oracle_reset(c);
        record_E(c, ah, 0, M);
        for (int m = 0; m < M; ++m) {
            step_once(c, m, 2);
            record_E(c, ah, m + 1, M);
        }
        /* Eq. (Gradient_FDTD) per owned sample, summed over the voxel's three samples, times dx^3 */
        const int shift = (align >> 1) & 1;   /* Etilde^{m+1/2} -> solver level m + shift */
        const double dV = c->g.dx * c->g.dx * c->g.dx;
        const int* b = c->g.design_box;
        for (int k = b[4]; k < b[5]; ++k)
            for (int j = b[2]; j < b[3]; ++j)
                for (int i = b[0]; i < b[1]; ++i) {
                    size_t v = design_index(c, i, j, k);
                    if (voxel_class(c, i, j, k) != 1) {
                        grad[v] = 0.0;
                        continue;
                    }
                    double rho = c->rho[v], g = 0.0;
                    for (int comp = 0; comp < 3; ++comp) {
                        const double* E = eh + ((size_t)comp * c->nd + v) * L;
                        const double* A = ah + ((size_t)comp * c->nd + v) * L;
                        double deps = c->m2.eps_inf[comp] - c->m1.eps_inf[comp];
                        double dsig = c->m2.sigma[comp] - c->m1.sigma[comp] + (1.0 - 2.0 * rho) * c->gamma;
                        double t1 = 0.0, t2 = 0.0, t3 = 0.0;
                        for (int m = 1; m <= M; ++m) {
                            int lp = m + shift, lm = m - 1 + shift;
                            double ap = lp <= M ? A[lp] : 0.0, am = lm >= 0 && lm <= M ? A[lm] : 0.0;
                            double e = E[M - m];
                            t1 += e * (ap - am);
                            t2 += e * 0.5 * (ap + am);
                            double dq = 0.0;
                            for (int p = 0; p < c->P[comp]; ++p) {
                                const cplx* q = qh[comp] + (v * (size_t)c->P[comp] + p) * L;
                                double dk = p < c->P1[comp] ? -1.0 : 1.0;   /* d kappa_1/d rho = -1, d kappa_2/d rho = +1 */
                                dq += dk * creal(q[M - m] - q[M - m + 1]);
                            }
                            /* the printed average of the two adjoint half-levels, or (align bit 2) the one
                             * level the eps_inf term's summation by parts pairs with this Q difference */
                            t3 += 2.0 * dq * ((align & 4) ? am : 0.5 * (ap + am));
                        }
                        g += -EPS0 * deps * t1 - dsig * t2 * c->dt + t3;
                    }
                    grad[v] = g * dV;
                }
    }
    for (int comp = 0; comp < 3; ++comp) free(qh[comp]);
    free(eh);
    free(ah);
    if (rc) return rc;
    if (F_out) *F_out = F;
    c->have_fwd = 0;     /* the DFT-mode forward state is not valid after paper mode */
    c->have_adj = 0;
    return 0;
}

/* ---------------------------------------------------------------------------------------------
 * Gradient.  With z = e^{j w dt}, the z-transform of the E update of a sample gives its discrete
 * admittance  Y(z) = (1/dt)[eps0 eps_inf (z-1) + sigma dt (z+1)/2 + sum_i kappa_i sum_p (z-1)(h_p + hb_p)],
 * h_p = beta_p (z+1)/(z-alpha_p), hb_p the same with conj(alpha_p), conj(beta_p) (the conjugate
 * pole of the pair).  Only eps_inf, sigma and kappa_i depend on rho (SI Eq. (InterpolatedModel);
 * a_p, c_p do not), so
 *   dY/drho = (1/dt)[eps0 (eps2-eps1)(z-1) + (sig2-sig1+(1-2 rho) gamma) dt (z+1)/2
 *                    + (z-1)(sum_{p in m2}(h+hb) - sum_{p in m1}(h+hb))],
 * the three terms of Eq. (Gradient_analytic) (eps_inf: first difference, sigma: average, poles:
 * first difference of Re Q, as in Eq. (Gradient_FDTD)).  With the adjoint DFT Lambda,
 *   dF/drho_v = - sum_{k owned by v} sum_f 2 Re{ dY_k/drho(w_f) Ehat_k(w_f) Lambda_k(w_f) },
 * and 0 on gap voxels (fixed air).  With one density per E sample (layout 1) the sum over k
 * collapses to the sample's own component.
 * ------------------------------------------------------------------------------------------- */
static cplx pair_response(cplx alpha, cplx beta, cplx z)
{
    return beta * (z + 1.0) / (z - alpha) + conj(beta) * (z + 1.0) / (z - conj(alpha));
}

int oracle_gradient(oracle_ctx* c, double* grad, size_t n)
{
    if (!c || !c->have_adj) return c ? fail(c, "gradient before adjoint") : 1;
    if (n != c->nvar) return fail(c, "gradient buffer size");
    const double dt = c->dt;
    memset(grad, 0, n * sizeof(double));
    for (int comp = 0; comp < 3; ++comp) {
        const int* b = c->sbox[comp];
        if (c->nd == 0) break;
        for (int k = b[4]; k < b[5]; ++k)
            for (int j = b[2]; j < b[3]; ++j)
                for (int i = b[0]; i < b[1]; ++i) {
                    if (!design_sample(c, comp, i, j, k)) continue;   /* gap: 0 */
                    size_t r = rho_index(c, comp, i, j, k), v = design_index(c, i, j, k);
                    double rho = c->rho[r];
                    for (int f = 0; f < c->g.n_freq; ++f) {
                        cplx z = cexp(I * 2.0 * M_PI * c->freqs[f] * dt);
                        cplx poles = 0.0;
                        for (int p = 0; p < c->P[comp]; ++p) {
                            cplx hp = pair_response(c->alpha[comp][p], c->beta[comp][p], z);
                            poles += (p < c->P1[comp]) ? -hp : hp;
                        }
                        cplx dY = (EPS0 * (c->m2.eps_inf[comp] - c->m1.eps_inf[comp]) * (z - 1.0)
                                   + (c->m2.sigma[comp] - c->m1.sigma[comp] + (1.0 - 2.0 * rho) * c->gamma) * dt * (z + 1.0) / 2.0
                                   + (z - 1.0) * poles) / dt;
                        size_t s = ((size_t)f * 3 + comp) * c->nd + v;
                        grad[r] += -2.0 * creal(dY * c->dft[0][s] * c->dft[1][s]);
                    }
                }
    }
    return 0;
}

int oracle_get_field(oracle_ctx* c, int which, double* dst, size_t n)
{
    if (!c || which < 0 || which > 5 || n != c->ncell) return 1;
    memcpy(dst, which < 3 ? c->E[which] : c->H[which - 3], n * sizeof(double));
    return 0;
}

int oracle_set_field(oracle_ctx* c, int which, const double* src, size_t n)
{
    if (!c || which < 0 || which > 5 || n != c->ncell) return 1;
    memcpy(which < 3 ? c->E[which] : c->H[which - 3], src, n * sizeof(double));
    return 0;
}

int oracle_get_dft(oracle_ctx* c, int adjoint, double* dst, size_t n_doubles)
{
    if (!c || n_doubles != 2 * (size_t)c->g.n_freq * 3 * c->nd) return 1;
    const cplx* d = c->dft[adjoint ? 1 : 0];
    for (size_t s = 0; s < n_doubles / 2; ++s) {
        dst[2 * s] = creal(d[s]);
        dst[2 * s + 1] = cimag(d[s]);
    }
    return 0;
}

int oracle_get_source(oracle_ctx* c, int which, double* dst, size_t n)
{
    const size_t M = (size_t)c->g.n_steps;
    if (which == 0 && n == M) memcpy(dst, c->src, M * sizeof(double));
    else if (which == 1 && n == M) { build_incident(c); memcpy(dst, c->einc, M * sizeof(double)); }
    else if (which == 2 && n == M) { build_incident(c); memcpy(dst, c->hinc, M * sizeof(double)); }
    else if (which == 3 && n == 3 * c->ngap * M) memcpy(dst, c->adjw, n * sizeof(double));
    else return 1;
    return 0;
}

/* Integer maps (bit-exact checks against the CUDA path):
 *  0: per E sample (3, nz, ny, nx): bits 0-1 voxel class (0 bg, 1 design, 2 gap), bit 2 PEC-fixed,
 *     bit 3 / bit 4: inside the CPML of the first / second derivative axis ((c+1)%3, (c+2)%3) at the
 *     sample's integer position, bit 5 forward dipole sample.
 *  1: per H sample (3, nz, ny, nx): bit 3 / bit 4 inside the CPML of derivative axis (c+1)%3 / (c+2)%3
 *     at the half-integer position.
 *  2: per voxel: design-box linear index or -1.     3: per voxel: gap linear index or -1. */
int oracle_get_index_map(oracle_ctx* c, int which, int32_t* dst, size_t n)
{
    const int nx = c->n[0], ny = c->n[1], nz = c->n[2];
    size_t need = (which <= 1) ? 3 * c->ncell : c->ncell;
    if (which < 0 || which > 3 || n != need) return 1;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t p = lin(c, i, j, k);
                int ijk[3] = {i, j, k};
                int cls = voxel_class(c, i, j, k);
                if (which == 2) { dst[p] = cls ? (int32_t)design_index(c, i, j, k) : -1; continue; }
                if (which == 3) { dst[p] = cls == 2 ? (int32_t)gap_index(c, i, j, k) : -1; continue; }
                for (int comp = 0; comp < 3; ++comp) {
                    int32_t v = 0;
                    for (int t = 0; t < 2; ++t) {
                        int a = (comp + 1 + t) % 3;
                        double u = ijk[a] + (which == 1 ? 0.5 : 0.0);
                        if (pml_depth(c->g.cpml[2 * a], c->g.cpml[2 * a + 1], c->n[a], u) > 0.0) v |= 1 << (3 + t);
                    }
                    if (which == 0) {
                        v |= cls == 2 ? 2 : design_sample(c, comp, i, j, k);
                        if (pec_fixed(c, comp, ijk)) v |= 4;
                        if (c->g.src_kind == 0 && comp == c->g.src_comp && i == c->g.src_pos[0] &&
                            j == c->g.src_pos[1] && k == c->g.src_pos[2]) v |= 32;
                    }
                    dst[(size_t)comp * c->ncell + p] = v;
                }
            }
    return 0;
}
