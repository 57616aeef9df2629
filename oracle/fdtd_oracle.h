/* Plain FP64 CPU oracle for one CCPR time-domain adjoint gradient evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load this library.  It shares no code, header, table or constant with the CUDA path.
 *
 * The oracle follows arXiv 2305.00234 step by step (equations named by their LaTeX labels):
 *   - CCPR permittivity, Eq. (CCPRModel), with the density blending of Eqs. (eps_mixed),
 *     (sigma_mixed), (Poles_mixed) (Methods, "Time-domain adjoint formulation"; SI Eq.
 *     (InterpolatedModel));
 *   - Maxwell + pole-current ADE system in the SI form, Eq. (Maxwells2);
 *   - Yee leapfrog ("FDTD implementation and design export") with a CPML boundary of
 *     configurable thickness ("Technical details of the optimization");
 *   - gap objective as the DFT |E|^2 at given frequencies, the frequency-domain form of
 *     Eq. (Objective_analyitically_enhancement); the adjoint run is the same solver driven at
 *     the gap by the time-reversed objective derivative (SI Eqs. (AlmostAdjoint),
 *     (Tranformations), (AdjointSystem)), which in the frequency domain is its conjugate;
 *   - gradient as the per-voxel correlation of forward and adjoint DFT fields with the density
 *     derivative of the discrete admittance, the three-term structure of Eq. (Gradient_analytic)
 *     and the difference/average structure of Eq. (Gradient_FDTD).
 *
 * Layout: every field array is (nz, ny, nx) with x fastest; voxel (i,j,k) owns E_x(i+1/2,j,k),
 * E_y(i,j+1/2,k), E_z(i,j,k+1/2).  Design-box arrays are (dnz, dny, dnx).  DFT arrays are
 * (F, 3, dnz, dny, dnx) complex, stored as interleaved (re, im) doubles.
 *
 * Density layouts.  0: one density per design voxel, shared by its three E samples.  1: one
 * density per E sample, as the discretisation of Sec. "FDTD implementation and design export"
 * counts them: the E_k samples lying in the closed design region are those of the voxels in the
 * design box extended by one on each +l face with l != k, N~_k = prod_l (N_l + 1 - delta_kl) of
 * them; the design variables are the three components' samples, concatenated (E_x, E_y, E_z),
 * each (z, y, x) with x fastest over its own extents.  With layout 1 the DFT arrays and the
 * design-box index map cover the design box grown by one cell on its +x, +y, +z sides; samples
 * there outside their component's set keep the background update.  Paper mode takes layout 0.
 */
#ifndef FDTD_ORACLE_H
#define FDTD_ORACLE_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct oracle_ctx oracle_ctx;

typedef struct {
    int nx, ny, nz;
    double dx;
    double courant;              /* dt = courant * dx / c0 */
    int n_steps;
    int cpml[6];                 /* thickness in cells on faces x-, x+, y-, y+, z-, z+ */
    double cpml_m, cpml_sigma_scale, cpml_kappa_max, cpml_a_max;
    int bc[3];                   /* 0 = PEC outer wall, 1 = periodic (then cpml must be 0) */
    int design_box[6];           /* half-open i0,i1,j0,j1,k0,k1 */
    int gap_box[6];              /* half-open, inside the design box; empty = all zero */
    int n_freq;
    const double* freqs_hz;
    const double* freq_weights;
    int src_kind;                /* 0 point dipole, 1 TF/SF plane wave along +x (E_z, H_y) */
    int src_comp;                /* dipole component 0,1,2 */
    int src_pos[3];              /* dipole voxel; for TF/SF src_pos[0] is the first total-field x index */
    double src_f0, src_fwhm_hz, src_t0, src_amp;
    double adj_tau;              /* envelope of the adjoint basis pulses (0: the source's) */
    const double* src_wave;      /* optional p(s dt/2), s = 0..2 n_steps, replacing the Gaussian pulse
                                    (copied at create) */
    int density_layout;          /* 0: one density per design voxel; 1: one per E sample (below) */
} oracle_grid_desc;

typedef struct {
    double eps_inf[3];
    double sigma[3];
    int n_poles[3];
    const double* a_re[3];
    const double* a_im[3];
    const double* c_re[3];
    const double* c_im[3];
} oracle_material;

/* Field selectors for oracle_get_field / oracle_set_field. */
enum { ORACLE_EX = 0, ORACLE_EY, ORACLE_EZ, ORACLE_HX, ORACLE_HY, ORACLE_HZ };

int oracle_create(const oracle_grid_desc* desc, oracle_ctx** out);
int oracle_set_materials(oracle_ctx* c, const oracle_material* bg, const oracle_material* m1,
                         const oracle_material* m2, double gamma);
int oracle_set_density(oracle_ctx* c, const double* rho, size_t n);
/* Resets the state to zero, runs n_steps with the forward source, accumulates the forward DFT
 * over the design box, returns the objective and (optionally) the gap DFT (F,3,gap) complex. */
int oracle_forward(oracle_ctx* c, double* F_out, double* gap_dft_out);
int oracle_adjoint(oracle_ctx* c);
int oracle_gradient(oracle_ctx* c, double* grad, size_t n);
/* Forward run plus its tangent-linear run in the density direction drho (n = design variables):
 * F and dF = d/de F(rho + e drho) at e = 0, the exact derivative of the discrete frequency-domain
 * objective, by forward-mode differentiation of the scheme; Ftd, dFtd the same for the time-domain
 * energy objective of paper mode.  Any output may be NULL.  Invalidates the forward/adjoint state. */
int oracle_tangent(oracle_ctx* c, const double* drho, size_t n, double* F_out, double* dF_out, double* Ftd_out,
                   double* dFtd_out);

/* Paper mode (tiny grids): the time-domain objective of Eq. (Objective_analyitically_enhancement),
 *   F_td = (eps0/2) dx^3 dt sum_{n=1..M} sum_{gap samples} (E^n)^2   (air in the gap),
 * from a forward run.  oracle_paper_gradient also runs the adjoint system of SI Eq. (AdjointSystem)
 * (the same solver, driven at the gap samples by the time-reversed functional derivative eps0 E)
 * and evaluates the paper's discrete gradient Eq. (Gradient_FDTD) from the stored forward E and Q
 * and adjoint E histories, times dx^3, per design voxel (the three owned samples share rho; gap
 * voxels 0).  The paper leaves the half-step alignment open: align bit 0 delays the adjoint drive
 * by one step (E^{M-m-1} instead of E^{M-m} at adjoint step m), bit 1 maps the adjoint levels
 * Etilde^{m +- 1/2} to the solver's Etilde^{m+1}, Etilde^{m} (else Etilde^{m}, Etilde^{m-1}); bit 2
 * pairs the pole term's Q difference with Etilde^{m-1/2} alone instead of the printed average of
 * Etilde^{m+1/2} and Etilde^{m-1/2}. */
int oracle_paper_objective(oracle_ctx* c, double* F_out);
int oracle_paper_gradient(oracle_ctx* c, int align, double* F_out, double* grad, size_t n);

/* Test hooks. */
int oracle_reset(oracle_ctx* c);
int oracle_step(oracle_ctx* c, int n_first, int n_count, int source_mode); /* 0 none 1 fwd 2 adj */
int oracle_get_field(oracle_ctx* c, int which, double* dst, size_t n);
int oracle_set_field(oracle_ctx* c, int which, const double* src, size_t n);
int oracle_get_dft(oracle_ctx* c, int adjoint, double* dst, size_t n_doubles);
int oracle_get_source(oracle_ctx* c, int which, double* dst, size_t n);   /* 0 dipole S(n+1/2),
                                         1 E_inc(n), 2 H_inc(n+1/2), 3 adjoint (gap sample, n) */
int oracle_get_index_map(oracle_ctx* c, int which, int32_t* dst, size_t n);
/* Single E sample of component comp blended at rho, driven by a prescribed curl sequence
 * (no spatial coupling): the same per-sample update routine the grid loop calls. */
int oracle_sample_response(oracle_ctx* c, int comp, double rho, int n, const double* curl,
                           double* e_out);
double oracle_dt(const oracle_ctx* c);
const char* oracle_last_error(const oracle_ctx* c);
void oracle_destroy(oracle_ctx* c);

#ifdef __cplusplus
}
#endif
#endif
