/* fdtd_ccpr.h — C-ABI of the GB300 (sm_103a) CCPR time-domain adjoint gradient library.
 *
 * One handle = one gradient problem for density-based topology optimisation with dispersive
 * materials (arXiv 2305.00234):
 *   forward 3-D Yee FDTD run with CPML and the CCPR pole-current ADE, the density rho in [0,1]
 *   blending two CCPR materials inside a design box (Methods, "Time-domain adjoint formulation",
 *   Eqs. (eps_mixed), (sigma_mixed), (Poles_mixed), (Maxwells)); running DFTs of E over the
 *   design box; a gap objective F = sum_f w_f sum_{gap samples} |Ehat(w_f)|^2 (frequency-domain
 *   form of Eq. (Objective_analyitically_enhancement)); the adjoint run, i.e. the same solver
 *   driven at the gap by the conjugated (time-reversed) objective derivative (SI Eq.
 *   (AdjointSystem)); and dF/drho per design voxel from the forward and adjoint DFTs (three-term
 *   structure of Eq. (Gradient_analytic), difference/average structure of Eq. (Gradient_FDTD)).
 *
 * Conventions (all calls):
 *  - Grid: nx*ny*nz cells, arrays (nz, ny, nx) with x fastest.  Voxel (i,j,k) owns E_x(i+1/2,j,k),
 *    E_y(i,j+1/2,k), E_z(i,j,k+1/2) (Yee layout, "FDTD implementation and design export"); those
 *    samples take the voxel's material and density.  Outer walls are PEC behind the CPML.
 *  - Time: dt = courant*dx/c0 (c0 = 299792458 m/s, mu0 = 1.25663706212e-6 H/m, eps0 =
 *    1/(mu0 c0^2)); E at integer steps, H at half steps; n_steps steps per run.
 *  - e^{j w t} convention (paper, below Eq. (CCPRModel)); DFT Ehat(w) = sum_{n=1..M} E^n e^{-j w n dt}.
 *  - Boxes are half-open [i0,i1)x[j0,j1)x[k0,k1) given as {i0,i1,j0,j1,k0,k1}.
 *  - Ownership: the library owns all device state.  Caller pointers are borrowed for the call
 *    only.  on_device = 1 means a device pointer valid on the handle's stream (the stream passed
 *    to fdtd_create_grid; NULL = the legacy default stream); 0 means a host pointer.
 *  - Errors: every call returns a status and never throws.  fdtd_last_error() gives the text.
 *    After FDTD_ERR_CUDA, FDTD_ERR_UNSTABLE or FDTD_ERR_TIMEOUT the handle accepts only
 *    fdtd_destroy, fdtd_last_error and fdtd_get_*.  A handle is not thread-safe; separate handles are.
 *  - Call order: create -> set_materials -> set_density -> forward -> adjoint -> gradient.
 *    set_materials/set_density invalidate earlier forward/adjoint results.
 */
#ifndef FDTD_CCPR_H
#define FDTD_CCPR_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct fdtd_ctx* fdtd_handle;

typedef enum {
    FDTD_OK = 0,
    FDTD_ERR_ARG = 1,       /* invalid argument or size mismatch */
    FDTD_ERR_OOM = 2,       /* device allocation failed */
    FDTD_ERR_CUDA = 3,      /* CUDA runtime error (handle is dead) */
    FDTD_ERR_STATE = 4,     /* calls out of order */
    FDTD_ERR_UNSTABLE = 5,  /* non-finite or exploding field detected (handle is dead) */
    FDTD_ERR_TIMEOUT = 6,   /* a bounded device wait gave up (handle is dead) */
    FDTD_ERR_CANCELLED = 7  /* cancelled by fdtd_cancel */
} fdtd_status;

/* Grid, time stepping, boxes, objective frequencies and source.
 *  cpml[6]: CPML thickness in cells on faces x-,x+,y-,y+,z-,z+ (the paper: 20 cells, "Technical
 *    details of the optimization"; profile parameters are not given there).  CFS-CPML with
 *    sigma = sigma_max d^m, kappa = 1+(kappa_max-1) d^m, a = a_max (1-d), d = depth fraction,
 *    sigma_max = cpml_sigma_scale * 0.8 (m+1)/(eta0 dx).
 *  precision: 32 (FP32 fields and pole currents) or 64 (all FP64).  DFT accumulators, the
 *    gradient and the coefficient precompute are FP64 in both.
 *  design_box must lie outside the CPML; gap_box inside design_box (gap voxels are fixed
 *    background material, gradient 0 there).
 *  density_layout 0: one density per design voxel, shared by the voxel's three E samples (E_x at
 *    (i+1/2, j, k), E_y at (i, j+1/2, k), E_z at (i, j, k+1/2)).  1: one density per E sample, the
 *    count of Sec. "FDTD implementation and design export": component k has
 *    N~_k = prod_l (N_l + 1 - delta_kl) samples (the design box's voxels extended by one on the +l
 *    faces, l != k), so the design variables are N~ = N~_x + N~_y + N~_z values, the three
 *    components' arrays concatenated, each (z, y, x) x fastest over its own extents.  With layout 1
 *    the working box (DFTs, index map 2) is the design box grown by one cell on its +x, +y, +z
 *    sides, and that box must lie outside the CPML; E samples of the working box outside their
 *    component's sample set, and gap samples, take the background update.  Paper mode
 *    (fdtd_paper_forward / fdtd_paper_gradient) takes layout 0 only.
 *  n_freq in [1, 8] objective frequencies (Hz) with weights.
 *  src_kind 0: soft point source on E_{src_comp} of voxel src_pos, drive added to (curl H) =
 *    src_amp (eps0/dt) p((n+1/2) dt);  src_kind 1: one-sided TF/SF plane wave along +x, E_z/H_y,
 *    first total-field plane x = src_pos[0] dx, incident field src_amp p(t) from a matched 1-D line.
 *    p(t) = exp(-(t-t0)^2/(2 tau^2)) sin(2 pi f0 (t-t0)), tau = sqrt(2 ln 2)/(pi src_fwhm_hz),
 *    t0 = src_t0 or 4 tau if src_t0 <= 0.
 *  src_wave: optional source waveform p(s dt/2), s = 0 .. 2 n_steps (2 n_steps + 1 doubles, copied
 *    during fdtd_create_grid), replacing the Gaussian pulse for either source kind (e.g. the
 *    paper's truncated sinc x Hanning window x carrier of Sec. "Optimization setup"); NULL: p above.
 *  adj_tau: envelope of the 2F adjoint basis pulses g(t){cos,sin}(w_f (t - 4 adj_tau));
 *    <= 0 selects the source's tau (then src_fwhm_hz > 0 is required even with src_wave). */
typedef struct {
    int nx, ny, nz;
    double dx;
    double courant;
    int n_steps;
    int cpml[6];
    double cpml_m, cpml_sigma_scale, cpml_kappa_max, cpml_a_max;
    int precision;
    int design_box[6];
    int gap_box[6];
    int n_freq;
    const double* freqs_hz;
    const double* freq_weights;
    int src_kind;
    int src_comp;
    int src_pos[3];
    double src_f0, src_fwhm_hz, src_t0, src_amp;
    double adj_tau;
    const double* src_wave;
    int density_layout;
} fdtd_grid_desc;

/* One CCPR material (Eq. (CCPRModel)): per Cartesian component k, eps_inf[k], sigma[k] (S/m)
 * and n_poles[k] pole pairs (a_p, c_p), each standing for c/(jw-a) + conj(c)/(jw-conj(a)); a in rad/s
 * with Re(a) <= 0 and a != 0, c in 1/s.  Arrays are read during the call only. */
typedef struct {
    double eps_inf[3];
    double sigma[3];
    int n_poles[3];
    const double* a_re[3];
    const double* a_im[3];
    const double* c_re[3];
    const double* c_im[3];
} fdtd_ccpr_material;

/* Per-kernel device time, measured with CUDA events on the handle's stream while profiling is on
 * (fdtd_set_profiling): one 16-step block in four is launched kernel by kernel between events,
 * the others as CUDA graphs.  *_ms sum and *_launches count those timed launches (grad: every
 * launch); launches counts every kernel this library launched since the last reset. */
typedef struct {
    /* summed device time per kernel: the background step's shell H update, fused interior update and
     * shell E update (one launch each per step), the E update inside the design box, the blocked
     * DFT, the gradient */
    double shell_h_ms, step_ms, shell_e_ms, ed_ms, dft_ms, grad_ms;
    long long shell_h_launches, step_launches, shell_e_launches, ed_launches, dft_launches, grad_launches;
    long long launches;                      /* every kernel launch of this library */
    /* algorithmic bytes per launch: each word the kernel must move, read once and written once */
    double bytes_shell_h_per_launch, bytes_step_per_launch, bytes_shell_e_per_launch, bytes_ed_per_launch,
        bytes_dft_per_launch, bytes_grad_per_launch;
    double dft_steps_per_launch;             /* time steps folded into one DFT launch */
    long long fused_step;                    /* 1: the grid has an interior box for the fused TMA kernel
                                                (x rows a multiple of 16 bytes, room inside the CPML);
                                                0: the shell kernels cover the whole grid */
    double interior_cells;                   /* cells of the interior box (one fused-kernel launch) */
    double interior_design_cells;            /* of which inside the working box (no E update there) */
    long long paired_shell;                  /* 1: the shell kernels update x-adjacent cell pairs (FP32, every
                                                x bound of the grid, the x CPML and the shell boxes even) */
    long long pdl_graphs;                    /* 1: the step graphs link each phase to the next through
                                                programmatic dependent launch edges; 0: ordinary edges */
    long long paired_design;                 /* 1: the design-E kernel updates x-adjacent sample pairs (FP32,
                                                up to 8 poles a component, nx and the working box's x origin
                                                and extent even) */
} fdtd_timings;

/* Create a problem on the given CUDA stream (cudaStream_t; NULL = default stream) of the current
 * device.  Validates the description and allocates every device buffer (footprint as returned
 * by fdtd_footprint_bytes).  Errors: FDTD_ERR_ARG (invalid desc), FDTD_ERR_OOM, FDTD_ERR_CUDA. */
fdtd_status fdtd_create_grid(const fdtd_grid_desc* desc, void* cuda_stream, fdtd_handle* out);

/* Paper mode: the paper's own objective and gradient, for comparison with the frequency-domain
 * ones above.  fdtd_paper_forward runs the forward system and returns the time-domain energy
 * objective of Eq. (Objective_analyitically_enhancement) over the gap,
 *   F = (eps0/2) dx^3 dt sum_{n=1..M} sum_{gap samples} (E^n)^2,
 * storing the full solver state every checkpoint_steps steps (<= 0: about sqrt(M x state / per-step
 * history), the memory-optimal interval) and the gap field at every step.  fdtd_paper_gradient then
 * evaluates Eq. (Gradient_FDTD) per design voxel (times dx^3; the voxel's three samples share rho; gap
 * voxels 0) by checkpoint-recompute: segment by segment from the last, the forward state is restored
 * and recomputed with the design-box E and pole-current term recorded, and the adjoint system of SI
 * Eq. (AdjointSystem) (the same solver on a second state set, driven at the gap samples by the
 * time-reversed functional derivative eps0 E) advances over the mirrored steps.  Readings of the
 * half-step alignment: the adjoint drive at adjoint step m is eps0 E^{M-m-1}, and the adjoint levels
 * m, m-1 stand for the paper's m+1/2, m-1/2.  pole_pairing 0 multiplies the pole term's
 * Re{Q^{M-m} - Q^{M-m+1}} by the printed average of those two levels, 1 by level m-1 alone.  With 1
 * the result is the exact gradient of the discrete objective once the fields and pole currents have
 * decayed within the window (as the derivation assumes); 0 approximates the pole term (closely for
 * Lorentz pairs, tens of percent off for a Drude pole).
 * Extra device memory: a second state set, one state checkpoint per segment and three
 * (checkpoint_steps + 1) x 3 x design-voxel history buffers.  grad: n = design voxels, dtype 0 float32
 * / 1 float64, on_device as for fdtd_gradient.  Errors: FDTD_ERR_ARG (no design box or gap; sizes),
 * FDTD_ERR_STATE (gradient before a paper forward, or after a density or material change),
 * FDTD_ERR_OOM, FDTD_ERR_UNSTABLE, FDTD_ERR_CUDA. */
fdtd_status fdtd_paper_forward(fdtd_handle h, int checkpoint_steps, double* F_out);
fdtd_status fdtd_paper_gradient(fdtd_handle h, int pole_pairing, void* grad, size_t n, int dtype, int on_device);

/* Device bytes a handle with this description and these pole counts would allocate
 * (p_total[k] = poles of m1 + m2 on component k).  For admission control; allocates nothing. */
fdtd_status fdtd_footprint_bytes(const fdtd_grid_desc* desc, const int p_total[3], size_t* bytes);

/* Materials: bg outside the design box and in the gap (must be non-dispersive: n_poles = 0);
 * m1 at rho = 0 and m2 at rho = 1 inside it (both materials' poles are kept, weighted 1-rho and
 * rho; Eq. (Poles_mixed)); gamma: conductivity damping rho(1-rho)gamma (Eq. (sigma_mixed)).
 * Pole coefficients alpha = e^{a dt}, beta = eps0 c (e^{a dt}-1)/(2a) are computed here in FP64.
 * Errors: FDTD_ERR_ARG (pole counts > 16 per component in total, Re a > 0, non-positive update
 * denominator at rho = 0 or 1). */
fdtd_status fdtd_set_materials(fdtd_handle h, const fdtd_ccpr_material* bg, const fdtd_ccpr_material* m1,
                               const fdtd_ccpr_material* m2, double gamma);

/* Density on the design box, (dnz, dny, dnx) x fastest, n = dnx*dny*dnz values in [0, 1] (with
 * density_layout 1: the N~ per-sample values described above; n_design of fdtd_get_info);
 * dtype 0 = float32, 1 = float64.  Values outside [0,1] or non-finite: FDTD_ERR_ARG (checked on
 * the device when on_device = 1). */
fdtd_status fdtd_set_density(fdtd_handle h, const void* rho, size_t n, int dtype, int on_device);

/* Forward run: zero state, n_steps steps with the forward source, forward DFT over the design
 * box.  F_out (host, nullable) receives the objective; gap_dft_out (host, nullable) receives the
 * gap DFT, (F, 3, gnz, gny, gnx) complex as interleaved (re, im) doubles.
 * Errors: FDTD_ERR_STATE before set_density, FDTD_ERR_UNSTABLE, FDTD_ERR_CUDA. */
fdtd_status fdtd_forward(fdtd_handle h, double* F_out, double* gap_dft_out);

/* Adjoint run (requires forward): builds the adjoint drive at every gap sample g as
 * sum_q r_{g,q} b_q(t) over the 2F basis pulses, r_g solving (2F x 2F, FP64 on the host)
 * sum_q r_{g,q} sum_{n<M} b_q((n+1/2)dt) e^{-j w_f n dt} = w_f conj(Ehat_g(w_f)), then runs the
 * same solver and accumulates the adjoint DFT. */
fdtd_status fdtd_adjoint(fdtd_handle h);

/* Gradient (requires adjoint): per design voxel
 *   dF/drho = -sum_{owned k} sum_f 2 Re{ dY_k/drho(w_f) Ehat_k(w_f) Lambda_k(w_f) },
 *   dY/drho = (1/dt)[eps0 d_eps (z-1) + (d_sigma + (1-2rho) gamma) dt (z+1)/2
 *                    + (z-1)(sum_{m2}(h+hb) - sum_{m1}(h+hb))],  z = e^{j w dt},
 *   h = beta (z+1)/(z-alpha), hb the same with conj(alpha), conj(beta); 0 on gap voxels.
 * With density_layout 1 the derivative is per E sample (one component k, dY_k/drho_k), in the
 * layout of fdtd_set_density, 0 on gap samples.
 * grad: n = n_design (fdtd_get_info), dtype 0 float32 / 1 float64, host or device.  grad_norm2_out
 * (nullable, host) receives sum of squares (FP64). */
fdtd_status fdtd_gradient(fdtd_handle h, void* grad, size_t n, int dtype, int on_device);
fdtd_status fdtd_gradient_norm(fdtd_handle h, double* grad_norm2_out);

/* Parity/inspection.  dst is a host buffer (on_device 0: the call waits for the copy) or a device
 * buffer (on_device 1: the copy is ordered on the handle's stream and the call does not wait).
 *  fdtd_get_field: which 0..5 = Ex,Ey,Ez,Hx,Hy,Hz after the last run, n = nx*ny*nz doubles (the field
 *    converted to FP64), (nz,ny,nx) x fastest.
 *  fdtd_get_dft: adjoint 0/1, n_doubles = 2*F*3*nd, layout (F,3,dnz,dny,dnx) complex interleaved over
 *    the working box (see density_layout).
 *  fdtd_get_index_map (host only, synchronous): which 0: (3,nz,ny,nx) per E sample: bits 0-1 voxel
 *    class (0 background, 1 design, 2 gap), bit 2 PEC-fixed, bits 3/4 inside the CPML of derivative
 *    axis (c+1)%3 / (c+2)%3 at the sample's integer position, bit 5 forward dipole sample;
 *    1: (3,nz,ny,nx) per H sample, bits 3/4 for half-integer positions; 2: per voxel design index
 *    or -1; 3: per voxel gap index or -1.  Computed on the device by the same index helpers the
 *    kernels use.
 *  fdtd_get_gradient_constants (host, after set_materials): the per-component, per-frequency
 *    constants of dY/drho = A + (1 - 2 rho) B (the derivative in fdtd_gradient), n_doubles = 12*F,
 *    layout [3][F] x (A.re, A.im, B.re, B.im): the dy_drho argument of fdtd_gradient_static.
 *  Errors: FDTD_ERR_ARG (sizes, which), FDTD_ERR_STATE (constants before set_materials). */
fdtd_status fdtd_get_field(fdtd_handle h, int which, double* dst, size_t n, int on_device);
fdtd_status fdtd_get_dft(fdtd_handle h, int adjoint, double* dst, size_t n_doubles, int on_device);
fdtd_status fdtd_get_index_map(fdtd_handle h, int which, int32_t* dst, size_t n);
fdtd_status fdtd_get_gradient_constants(fdtd_handle h, double* dst, size_t n_doubles);

/* Failure-path test hook (not part of the method).  With timeout_ns > 0, every later run has block
 * (0, 0, 0) of the interior step kernel wait at step 0, for timeout_ns, on an mbarrier that no copy
 * completes; the wait runs out, the block records it in the handle's device flags, waits for its own
 * copies in flight (bounded) and returns, later blocks skip their work, and the run returns
 * FDTD_ERR_TIMEOUT; the handle is dead afterwards.  Nothing faults: the device context stays usable
 * for other handles.  timeout_ns = 0 turns the hook off.  Errors: FDTD_ERR_ARG (a grid without an
 * interior box, where the step kernel does not run; timeout_ns outside [0, 1e10]). */
fdtd_status fdtd_inject_wait_timeout(fdtd_handle h, long long timeout_ns);

/* Profiling: when on, runs time a sample of their kernel launches with CUDA events (see
 * fdtd_timings); fdtd_get_timings returns the sums since fdtd_reset_timings. */
fdtd_status fdtd_set_profiling(fdtd_handle h, int on);
fdtd_status fdtd_get_timings(fdtd_handle h, fdtd_timings* out);
fdtd_status fdtd_reset_timings(fdtd_handle h);

/* Scalars: dt (s), design variable count (voxels, or N~ with density_layout 1), gap voxel count,
 * device footprint (bytes). */
fdtd_status fdtd_get_info(fdtd_handle h, double* dt, size_t* n_design, size_t* n_gap, size_t* device_bytes);

/* Request that a run in progress on another host thread stop at the next chunk boundary
 * (it returns FDTD_ERR_CANCELLED).  The only call that may come from another thread. */
fdtd_status fdtd_cancel(fdtd_handle h);

/* Gradient for callers that cannot allocate device memory.  Some hosts own all device memory
 * themselves (a framework that has reserved it for its pool allocator, a plug-in host that forbids
 * its plug-ins to allocate), and some loops cannot afford the device-wide synchronisation that
 * cudaMalloc/cudaFree imply; such callers keep the forward and adjoint DFTs in their own buffers
 * and call this instead of fdtd_gradient.  It computes the same per-voxel dF/drho and squared norm
 * from caller-owned device buffers and allocates nothing: its scratch (per-block partial sums, a
 * completion counter and the dY/drho constants) is a 1 MiB static array in device memory, which
 * every GPU that loads this library holds until the process exits.  The paper has no counterpart;
 * this is a calling convention, not part of the method.
 *  It takes one density per design voxel (density_layout 0 of fdtd_grid_desc): the DFTs span
 *    exactly the design box and the three samples of a voxel share its rho.
 *  dft_fwd, dft_adj: device, (n_freq, 3, dnz, dny, dnx) complex as interleaved (re, im) doubles over
 *    design_box (what fdtd_get_dft returns for a density_layout 0 handle); rho: device, design-box
 *    densities, rho_dtype 0 float32 / 1 float64; design_box, gap_box (nullable): host, half-open,
 *    gap voxels get 0; dy_drho: host, [3][n_freq] x (A.re, A.im, B.re, B.im) with
 *    dY/drho = A + (1 - 2 rho) B (fdtd_get_gradient_constants of the handle that ran the DFTs);
 *    grad: device, one double per design voxel (output); grad_norm2: host, nullable (output; when
 *    given, the call waits for the stream); cuda_stream: cudaStream_t or NULL.
 *  Limits: n_freq <= 8 and at most 33,513,216 design voxels (the partial sums must fit the
 *    scratch); beyond them FDTD_ERR_ARG with the reason in fdtd_last_error(NULL).
 *  The first call on each device looks up the scratch array's device address with that device
 *    current; make that first call before any stream capture.  All calls share the one array and
 *    it keeps the previous call's contents (each call clears its counter itself): calls that
 *    overlap on the GPU, from several threads or streams, race and must be serialised. */
fdtd_status fdtd_gradient_static(const double* dft_fwd, const double* dft_adj, const void* rho, int rho_dtype,
                                 const int design_box[6], const int gap_box[6], int n_freq,
                                 const double* dy_drho, double* grad, double* grad_norm2, void* cuda_stream);

/* Density filter and projection on a design-box array (Sec. "Filtering and projection"):
 *   rho_t = Eq. (FilterFunction): the cone-weighted mean of rho over the sphere |r_m - r_n| < R,
 *           weight w = R - |r_m - r_n| (distances in voxels), neighbourhoods cut at the box faces;
 *   rho_b = Eq. (Projection): (tanh(beta eta) + tanh(beta (rho_t - eta))) / (tanh(beta eta) + tanh(beta (1 - eta))).
 * rho, rho_t, rho_b: device float32 arrays (nz, ny, nx), x fastest; R in (0, 12] voxels, beta > 0,
 * eta in [0, 1]; work is ordered on cuda_stream (temporary buffers come from the stream-ordered
 * allocator).  Errors: FDTD_ERR_ARG, text in fdtd_last_error(NULL). */
fdtd_status fdtd_filter_project(const float* rho, float* rho_t, float* rho_b, int nx, int ny, int nz, double R,
                                double beta, double eta, void* cuda_stream);

/* Chain rule through filter and projection, Eq. (GradientsFiltered): dF/drho[n] =
 * sum_m dF/drho_b[m] (d rho_b/d rho_t)[m] w(m,n) / sum_k w(m,k), from rho_t of fdtd_filter_project and
 * dF/drho_b (e.g. fdtd_gradient's output).  Same layout and limits as fdtd_filter_project. */
fdtd_status fdtd_filter_project_grad(const float* rho_t, const float* dF_drho_b, float* dF_drho, int nx, int ny,
                                     int nz, double R, double beta, double eta, void* cuda_stream);

/* Batches: several runs (forward or adjoint runs of different handles, different grid sizes) advanced
 * together by one persistent kernel, for serving many gradient evaluations at once.  The paper has no
 * counterpart; the arithmetic of a batched run is the method's (the same cell updates, pole recursion and
 * DFT as fdtd_forward / fdtd_adjoint; the background cells take the per-cell kernels' rounding instead
 * of the fused interior kernel's, so results agree with fdtd_forward to FP32 rounding, and a run's results
 * do not depend on which other runs share its launches).
 *  Each launch is one CUDA graph (zero the work counter, the persistent kernel) whose kernel takes work
 *  items (one phase, H or E, of one step of one run, on 4-8 z planes x 256-1024 (x, y) columns) from a global
 *  counter in an order where every item only waits for items numbered before it; every wait is bounded.
 *  fdtd_batch_create: on the current device; work is ordered after cuda_stream (NULL: legacy default
 *    stream) at each fdtd_batch_run and the stream waits for it afterwards.
 *  fdtd_batch_submit: adjoint 0 starts the handle's forward run (after set_materials and set_density),
 *    adjoint 1 its adjoint run (after a forward run, batched or not; the drive is built as in
 *    fdtd_adjoint).  At most 16 runs at a time; FP32 handles on the batch's device only.  Until the run
 *    ends, calls on the handle other than fdtd_get_*, fdtd_last_error and fdtd_destroy (which removes
 *    the run) return FDTD_ERR_STATE.
 *  fdtd_batch_run: one launch advancing every submitted run by up to max_steps steps; returns the
 *    handles whose runs ended in done[0 .. *n_done) with their status (FDTD_OK, or FDTD_ERR_UNSTABLE /
 *    FDTD_ERR_CUDA for that handle alone); capacity must be at least the number of runs in the batch.
 *    A finished forward run leaves the handle as fdtd_forward does (fdtd_get_objective gives F and the
 *    gap DFT); a finished adjoint run as fdtd_adjoint does (fdtd_gradient next).  If a wait of the
 *    persistent kernel gives up: FDTD_ERR_TIMEOUT, and the batch and its handles are dead.
 *  fdtd_batch_set_wait_limit: the limit of one wait (default 1 s); gate = 1 is a failure-path test hook
 *    that makes the first work item also wait on a flag nothing sets, so that the next fdtd_batch_run
 *    returns FDTD_ERR_TIMEOUT without any GPU fault.
 *  fdtd_batch_set_blocks: blocks of the persistent launches (0, the default: as many as fit on the
 *    device; fewer leave SMs to other work on the device, e.g. runs outside the batch).
 *  fdtd_batch_info: runs in the batch and launches made.
 *  Errors: FDTD_ERR_ARG, FDTD_ERR_STATE (call order, full batch, dead batch), FDTD_ERR_OOM,
 *  FDTD_ERR_TIMEOUT, FDTD_ERR_CUDA; the text of batch calls is in fdtd_last_error(NULL). */
typedef struct fdtd_batch_ctx* fdtd_batch;
fdtd_status fdtd_batch_create(void* cuda_stream, fdtd_batch* out);
fdtd_status fdtd_batch_submit(fdtd_batch b, fdtd_handle h, int adjoint);
fdtd_status fdtd_batch_run(fdtd_batch b, int max_steps, fdtd_handle* done, fdtd_status* done_status, int capacity,
                           int* n_done);
fdtd_status fdtd_batch_set_wait_limit(fdtd_batch b, long long wait_ns, int gate);
fdtd_status fdtd_batch_set_blocks(fdtd_batch b, int blocks);
fdtd_status fdtd_batch_info(fdtd_batch b, int* n_runs, long long* launches);
fdtd_status fdtd_batch_destroy(fdtd_batch b);

/* Objective of the handle's last forward run (fdtd_forward or a batched forward run): F_out (host,
 * nullable) and the gap DFT (host, nullable, as fdtd_forward's gap_dft_out).  FDTD_ERR_STATE before a
 * forward run. */
fdtd_status fdtd_get_objective(fdtd_handle h, double* F_out, double* gap_dft_out);

/* Message of the handle's last failed call; with h = NULL, of the calling thread's last failed
 * call (fdtd_create_grid and fdtd_footprint_bytes have no handle to report through). */
const char* fdtd_last_error(fdtd_handle h);
fdtd_status fdtd_destroy(fdtd_handle h);

#ifdef __cplusplus
}
#endif
#endif
