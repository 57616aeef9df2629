// Host implementation of the C-ABI declared in include/fdtd_ccpr.h.
//
// Everything that is not per-cell work happens here in FP64 on the host, once per call:
// CPML profiles, CCPR pole coefficients alpha = e^{a dt}, beta = eps0 c (e^{a dt}-1)/(2a),
// update denominators, source waveforms (including the matched 1-D line of the TF/SF plane
// wave), DFT phase tables, the 2F x 2F adjoint basis solve and the gradient constants
// dY/drho(w_f).  The per-cell work runs in the kernels of fdtd_kernels.cuh.
//
// A run enqueues CUDA graphs of up to kGraphSteps (H, E) step pairs on a private stream; the
// caller's stream is fenced with events before and after, so device pointers passed with
// on_device = 1 are ordered with the caller's work.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "fdtd_ccpr.h"
#include "fdtd_launch.h"

namespace {

using cd = std::complex<double>;
using fdtd::cpx;
using fdtd::DParams;
using fdtd::GParams;
using fdtd::KParams;
using fdtd::PoleTable;
using fdtd::StepMaps;
using fdtd::kSX;
using fdtd::kSYE;
using fdtd::kSYH;

constexpr double kC0 = 299792458.0;
constexpr double kMu0 = 1.25663706212e-6;
const double kEps0 = 1.0 / (kMu0 * kC0 * kC0);
const double kPi = 3.14159265358979323846;
constexpr int kGraphSteps = fdtd::kMaxSnap;   // one DFT block per captured graph
constexpr int kChunkSteps = 512;
constexpr int kProfEvery = 4;                  // profiling times one DFT block in four

struct Err {
    fdtd_status code;
    std::string msg;
};

#define CK(call)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) throw Err{FDTD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

[[noreturn]] void arg_error(const std::string& m) { throw Err{FDTD_ERR_ARG, m}; }

// e^{z} - 1 without cancellation for small |z|.
cd expm1c(cd z)
{
    const double x = z.real(), y = z.imag();
    const double s = std::sin(0.5 * y);
    return cd(std::expm1(x) * std::cos(y) - 2.0 * s * s, std::exp(x) * std::sin(y));
}

struct Pole {
    cd a, c;
};

struct Material {
    double eps[3] = {1, 1, 1}, sig[3] = {0, 0, 0};
    std::vector<Pole> poles[3];
};

Material import_material(const fdtd_ccpr_material* m, const char* what)
{
    if (!m) arg_error(std::string(what) + ": null material");
    Material out;
    for (int k = 0; k < 3; ++k) {
        out.eps[k] = m->eps_inf[k];
        out.sig[k] = m->sigma[k];
        if (!std::isfinite(out.eps[k]) || !std::isfinite(out.sig[k])) arg_error(std::string(what) + ": non-finite eps/sigma");
        if (m->n_poles[k] < 0 || m->n_poles[k] > fdtd::kMaxPoles) arg_error(std::string(what) + ": bad pole count");
        for (int p = 0; p < m->n_poles[k]; ++p) {
            Pole q{cd(m->a_re[k][p], m->a_im[k][p]), cd(m->c_re[k][p], m->c_im[k][p])};
            if (!(q.a.real() <= 0.0) || q.a == cd(0.0, 0.0)) arg_error(std::string(what) + ": pole with Re(a) > 0 or a = 0");
            if (!std::isfinite(q.c.real()) || !std::isfinite(q.c.imag())) arg_error(std::string(what) + ": non-finite residue");
            out.poles[k].push_back(q);
        }
    }
    return out;
}

// Work-item shape of a batched run: z planes sz and (x, y) columns cw per item.  Small grids take small
// items (more of them in flight, fewer planes marched by each thread), large grids large ones (less
// per-item overhead).
void batch_shape(const fdtd_grid_desc& d, int* sz, int* cw)
{
    const long long nxy = (long long)d.nx * d.ny;
    *sz = nxy * d.nz >= (1LL << 21) ? 2 * fdtd::kMinBatchSZ : fdtd::kMinBatchSZ;
    *cw = nxy >= 32768 ? 4 * fdtd::kBatchThreads : fdtd::kBatchThreads;
#ifdef FDTD_BATCH_SZ
    *sz = FDTD_BATCH_SZ;
#endif
#ifdef FDTD_BATCH_CW
    *cw = FDTD_BATCH_CW;
#endif
}

// CFS-CPML coefficients at position u (cells) along an axis of n cells with lo/hi layers.
void pml_point(const fdtd_grid_desc& d, double dt, int lo, int hi, int n, double u, double* kinv, double* b, double* c)
{
    double depth = 0.0;
    if (lo > 0 && u < lo)
        depth = (lo - u) / lo;
    else if (hi > 0 && u > n - hi)
        depth = (u - (n - hi)) / hi;
    if (depth <= 0.0) {
        *kinv = 1.0;
        *b = 1.0;
        *c = 0.0;
        return;
    }
    const double eta0 = kMu0 * kC0;
    const double smax = d.cpml_sigma_scale * 0.8 * (d.cpml_m + 1.0) / (eta0 * d.dx);
    const double gm = std::pow(depth, d.cpml_m);
    const double sig = smax * gm;
    const double kap = 1.0 + (d.cpml_kappa_max - 1.0) * gm;
    const double al = d.cpml_a_max * (1.0 - depth);
    *kinv = 1.0 / kap;
    *b = std::exp(-(sig / kap + al) * dt / kEps0);
    *c = sig > 0.0 ? sig * (*b - 1.0) / (sig * kap + kap * kap * al) : 0.0;
}

double src_tau(const fdtd_grid_desc& d) { return std::sqrt(2.0 * std::log(2.0)) / (kPi * d.src_fwhm_hz); }

// Source waveform at t (a multiple of dt/2): the caller's samples if given, else the Gaussian pulse.
double src_pulse(const fdtd_grid_desc& d, double dt, double t)
{
    if (d.src_wave) {
        const long s = std::lround(2.0 * t / dt);
        return (s >= 0 && s <= 2L * d.n_steps) ? d.src_wave[s] : 0.0;
    }
    const double tau = src_tau(d);
    const double t0 = d.src_t0 > 0.0 ? d.src_t0 : 4.0 * tau;
    const double x = t - t0;
    return std::exp(-x * x / (2.0 * tau * tau)) * std::sin(2.0 * kPi * d.src_f0 * x);
}

bool box_empty(const int* b) { return b[1] <= b[0] || b[3] <= b[2] || b[5] <= b[4]; }

long long box_count(const int* b) { return box_empty(b) ? 0 : (long long)(b[1] - b[0]) * (b[3] - b[2]) * (b[5] - b[4]); }

// Working box of the solver: the design box, or with the per-sample density layout the design box
// grown by one cell on its +x, +y, +z sides (the component sample boxes are inside it).
void working_box(const fdtd_grid_desc& d, int out[6])
{
    std::memcpy(out, d.design_box, 6 * sizeof(int));
    if (d.density_layout == 1 && !box_empty(out))
        for (int a = 0; a < 3; ++a) out[2 * a + 1] += 1;
}

// Design variables: voxels (layout 0) or sum_k prod_l (N_l + 1 - delta_kl) samples (layout 1);
// off[c] is where component c's samples start, md[c] their (x, y, z) extents.
size_t design_vars(const fdtd_grid_desc& d, long long off[4], int md[3][3])
{
    const int* db = d.design_box;
    const int N[3] = {db[1] - db[0], db[3] - db[2], db[5] - db[4]};
    off[0] = 0;
    for (int c = 0; c < 3; ++c) {
        long long cnt = 1;
        for (int a = 0; a < 3; ++a) {
            md[c][a] = box_empty(db) ? 0 : N[a] + (d.density_layout == 1 && a != c ? 1 : 0);
            cnt *= md[c][a];
        }
        off[c + 1] = off[c] + cnt;
    }
    if (d.density_layout != 1) return (size_t)box_count(db);
    return (size_t)off[3];
}

void validate(const fdtd_grid_desc& d)
{
    const int n[3] = {d.nx, d.ny, d.nz};
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 4 || n[a] > 65535) arg_error("grid axis size out of [4, 65535]");
        if (d.cpml[2 * a] < 0 || d.cpml[2 * a + 1] < 0 || d.cpml[2 * a] + d.cpml[2 * a + 1] > n[a] - 2)
            arg_error("bad CPML thickness");
    }
    if ((long long)d.nx * d.ny * d.nz > (1LL << 31) - 1) arg_error("grid larger than 2^31 cells");
    if (!(d.dx > 0.0) || !(d.courant > 0.0) || !(d.courant <= 1.0 / std::sqrt(3.0) + 1e-12))
        arg_error("dx must be > 0 and 0 < courant <= 1/sqrt(3)");
    if (d.n_steps < 1) arg_error("n_steps must be >= 1");
    if (d.precision != 32 && d.precision != 64) arg_error("precision must be 32 or 64");
    if (d.n_freq < 1 || d.n_freq > fdtd::kMaxFreq || !d.freqs_hz) arg_error("n_freq must be in [1, 8]");
    for (int f = 0; f < d.n_freq; ++f)
        if (!(d.freqs_hz[f] > 0.0) || (d.freq_weights && !std::isfinite(d.freq_weights[f]))) arg_error("bad frequency/weight");
    if (!(d.cpml_m >= 0.0) || !(d.cpml_kappa_max >= 1.0) || !(d.cpml_a_max >= 0.0) || !(d.cpml_sigma_scale >= 0.0))
        arg_error("bad CPML profile parameters");
    if (d.density_layout != 0 && d.density_layout != 1) arg_error("density_layout must be 0 (per voxel) or 1 (per E sample)");
    int db[6];
    working_box(d, db);
    const int* gb = d.gap_box;
    if (!box_empty(db)) {
        for (int a = 0; a < 3; ++a)
            if (db[2 * a] < d.cpml[2 * a] || db[2 * a + 1] > n[a] - d.cpml[2 * a + 1] || db[2 * a] >= db[2 * a + 1])
                arg_error(d.density_layout == 1 ? "design box grown by one cell on its +x/+y/+z sides must lie inside the grid and outside the CPML"
                                                : "design box must lie inside the grid and outside the CPML");
        if (box_count(db) > (1LL << 31) - 1) arg_error("design box too large");
        if (3LL * (db[5] - db[4]) > 65535) arg_error("design box spans more than 21845 z planes");
    }
    if (!box_empty(gb)) {
        if (box_empty(db)) arg_error("gap box without a design box");
        for (int a = 0; a < 3; ++a)
            if (gb[2 * a] < d.design_box[2 * a] || gb[2 * a + 1] > d.design_box[2 * a + 1])
                arg_error("gap box must lie inside the design box");
    }
    if (d.src_kind == 0) {
        for (int a = 0; a < 3; ++a)
            if (d.src_pos[a] < 0 || d.src_pos[a] >= n[a]) arg_error("dipole outside the grid");
        if (d.src_comp < 0 || d.src_comp > 2) arg_error("bad dipole component");
    } else if (d.src_kind == 1) {
        if (d.src_pos[0] < d.cpml[0] + 1 || d.src_pos[0] >= d.nx - d.cpml[1]) arg_error("TF/SF plane must lie outside the x CPML");
    } else {
        arg_error("src_kind must be 0 (dipole) or 1 (TF/SF plane)");
    }
    if (!std::isfinite(d.src_amp)) arg_error("bad source amplitude");
    if (!d.src_wave && (!(d.src_fwhm_hz > 0.0) || !(d.src_f0 >= 0.0))) arg_error("bad source parameters");
    if (!(d.adj_tau > 0.0) && !(d.src_fwhm_hz > 0.0)) arg_error("adjoint pulses need adj_tau > 0 or src_fwhm_hz > 0");
    if (d.src_wave)
        for (long s = 0; s <= 2L * d.n_steps; ++s)
            if (!std::isfinite(d.src_wave[s])) arg_error("non-finite source waveform sample");
}

size_t footprint(const fdtd_grid_desc& d, const int ptot[3])
{
    const size_t ts = d.precision == 64 ? 8 : 4;
    const size_t ncell = (size_t)d.nx * d.ny * d.nz;
    int wb[6];
    working_box(d, wb);
    const size_t nd = (size_t)box_count(wb);
    long long off[4];
    int md[3][3];
    const size_t nvar = design_vars(d, off, md);
    const size_t nv = std::max(nd, nvar);
    const size_t ng = (size_t)box_count(d.gap_box);
    const int n[3] = {d.nx, d.ny, d.nz};
    const size_t cs = (ncell + 31) / 32 * 32;
    size_t b = 4 * 3 * cs * ts;                                       // E, H: two buffers each
    for (int a = 0; a < 3; ++a) {                                     // psi: 2 E + 2 H components per axis
        const size_t w = (size_t)d.cpml[2 * a] + d.cpml[2 * a + 1];
        b += 6 * (ncell / n[a]) * w * ts + 8 * w * ts;               // psi_E, psi_H (two buffers)
    }
    b += (d.density_layout == 1 ? 3 : 1) * nd * ts;                  // rho (per component with layout 1)
    for (int k = 0; k < 3; ++k) b += nd * (size_t)ptot[k] * 2 * ts;   // Q
    b += 2 * nd * 3 * (size_t)d.n_freq * 16;                          // forward + adjoint DFT
    b += (size_t)fdtd::kMaxSnap * 3 * nd * ts + nv * 8;               // DFT snapshot ring, staging
    b += nv * 8 + ((nv + 255) / 256 + 1) * 8;                         // gradient + partials
    b += ((size_t)d.n_steps + 1) * d.n_freq * 2 * ts;                 // phase table
    b += (size_t)d.n_steps * (2 * fdtd::kMaxBasis + 2) * ts;          // source waves, TF/SF tables
    b += (ng * 3 * fdtd::kMaxBasis + 3) * ts + ng * 3 * d.n_freq * 16;
    b += sizeof(PoleTable<double>) + 256;
    return b;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (no libcuda link).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    });
    return fn;
}

// Library-private stream-ordered memory pool per device.  Handles allocate and free on their own
// stream, so creating or destroying one never synchronises the device (cudaFree does), and freed
// memory stays in the pool for the next handle instead of going back to the driver.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pool[kMaxDevices] = {};

cudaMemPool_t device_pool(int device)
{
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (device < 0 || device >= kMaxDevices) throw Err{FDTD_ERR_ARG, "device ordinal above 63"};
    if (!g_pool[device]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t pool = nullptr;
        CK(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = ~0ull;
        CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        g_pool[device] = pool;
    }
    return g_pool[device];
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Typed solver
// ---------------------------------------------------------------------------------------------
struct SolverBase {
    virtual ~SolverBase() = default;
    virtual void interior_box(int ib[6]) const = 0;
    virtual bool has_interior() const = 0;
    virtual bool paired_shell() const = 0;
    virtual bool pdl_graphs() const = 0;
    virtual bool paired_design() const = 0;
};

struct fdtd_ctx {
    fdtd_grid_desc d{};
    std::vector<double> freqs, weights, wave;
    cudaStream_t user = nullptr, work = nullptr;
    cudaStream_t side = nullptr;                       // second branch of the captured step graph
    cudaEvent_t fence = nullptr, fork = nullptr, join = nullptr;
    int device = 0;
    double dt = 0;
    size_t ncell = 0, nd = 0, ngap = 0;    // nd: working-box voxels
    size_t nvar = 0;                    // design variables (nd, or the per-sample count with layout 1)
    long long voff[4] = {0, 0, 0, 0};  // layout 1: offsets of the components' samples
    int vdim[3][3] = {};               //           and their (x, y, z) extents
    int dbu[6] = {0, 0, 0, 0, 0, 0};   // the caller's design box
    int dn[3] = {0, 0, 0}, gn[3] = {0, 0, 0};
    bool has_mat = false, has_rho = false, has_fwd = false, has_adj = false, has_grad = false, dead = false;
    double F_last = 0.0;                // objective of the last forward run
    struct fdtd_batch_ctx* batch = nullptr;   // the batch running one of this handle's runs, if any
    int batch_slot = -1;
    cudaEvent_t bfence = nullptr;       // orders the handle's stream before the batch's
    std::string err;
    std::atomic<int> cancel{0};
    size_t bytes = 0;
    std::vector<void*> allocs;
    // profiling
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    fdtd_timings tim{};
    std::unique_ptr<SolverBase> impl;

    void* alloc(size_t n)
    {
        void* p = nullptr;
        if (n == 0) n = 16;
        n = (n + 255) & ~size_t(255);
        if (cudaMallocFromPoolAsync(&p, n, device_pool(device), work) != cudaSuccess) {
            cudaGetLastError();
            throw Err{FDTD_ERR_OOM, "device allocation of " + std::to_string(n) + " bytes failed"};
        }
        allocs.push_back(p);
        bytes += n;
        return p;
    }
    void free_all()
    {
        for (void* p : allocs) cudaFreeAsync(p, work);
        allocs.clear();
    }
};

template <typename T>
struct Solver : SolverBase {
    fdtd_ctx* c;
    KParams<T> base{};              // shared part of the kernel parameters
    KParams<T> pf{}, pa{};          // forward / adjoint
    T* src_r[2] = {nullptr, nullptr};
    T* src_wave[2] = {nullptr, nullptr};
    T* einc = nullptr;
    T* hinc = nullptr;
    T* rho = nullptr;
    PoleTable<T>* poles = nullptr;
    PoleTable<T> htab{};            // the same table, passed by value to the design-E kernel
    double2* dft[2] = {nullptr, nullptr};
    using V2 = typename fdtd::vec2_of<T>::type;
    V2* phase = nullptr;
    T* snap = nullptr;
    void* staging = nullptr;
    DParams<T> dp[2]{};             // forward / adjoint DFT kernel parameters
    int bucket = 16;
    double2* gapbuf = nullptr;
    double2* AB = nullptr;
    double* grad = nullptr;
    double* partial = nullptr;
    unsigned* counter = nullptr;
    int* ctl = nullptr;
    int ptot[3] = {0, 0, 0};
    bool fused = false;             // an interior box for the fused TMA step kernel exists
    bool use_pdl = true;            // step graphs with programmatic edges between phases (else captured)
    bool pdl_built = false;         // a step graph with programmatic edges has been instantiated
    StepMaps maps[2]{};             // tensor maps of the buffers read by even / odd steps
    fdtd::ShellBoxes shell{};       // the cells around the interior box
    std::vector<double2> ab_host;
    std::vector<double> gap_dft;     // host copy of the forward gap DFT, (f,c,gv) complex
    double adj_cond = 0.0;
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [mode][full, remainder]

    explicit Solver(fdtd_ctx* ctx) : c(ctx) {}
    void interior_box(int ib[6]) const override { std::copy(base.ib, base.ib + 6, ib); }
    bool has_interior() const override { return fused; }
    bool paired_shell() const override { return shell.pair != 0; }
    bool pdl_graphs() const override { return use_pdl && pdl_built; }
    bool paired_design() const override { return base.ed_pair != 0; }
    ~Solver() override
    {
        for (auto& g : graph)
            for (auto& x : g)
                if (x) cudaGraphExecDestroy(x);
    }

    T* talloc(size_t n) { return (T*)c->alloc(n * sizeof(T)); }

    void allocate(const int p_total[3])
    {
        const fdtd_grid_desc& d = c->d;
        KParams<T>& p = base;
        p.nx = d.nx;
        p.ny = d.ny;
        p.nz = d.nz;
        p.plane = (long long)d.nx * d.ny;
        p.ncell = p.plane * d.nz;
        std::memcpy(p.db, d.design_box, sizeof p.db);
        std::memcpy(p.gb, d.gap_box, sizeof p.gb);
        if (box_empty(p.db)) std::fill(p.db, p.db + 6, 0);
        if (box_empty(p.gb)) std::fill(p.gb, p.gb + 6, 0);
        p.dnx = c->dn[0];
        p.dny = c->dn[1];
        p.dplane = (long long)c->dn[0] * c->dn[1];
        p.nd = (long long)c->nd;
        p.gnx = c->gn[0];
        p.gny = c->gn[1];
        p.gplane = (long long)c->gn[0] * c->gn[1];
        const int n[3] = {d.nx, d.ny, d.nz};
        for (int a = 0; a < 3; ++a) {
            p.cpl[a] = d.cpml[2 * a];
            p.cph[a] = d.cpml[2 * a + 1];
            p.W[a] = p.cpl[a] + p.cph[a];
        }
        // Each field is one block of three components, component stride cs (a multiple of 32 elements),
        // so that one 4-D tensor map covers it.  A step reads one buffer of each pair and writes the other.
        split_grid(p);
        cs = ((size_t)c->ncell + 31) / 32 * 32;
        T* fld[4];
        for (int f = 0; f < 4; ++f) fld[f] = talloc(3 * cs);
        for (int cc = 0; cc < 3; ++cc) {
            p.E[cc] = fld[0] + cc * cs;
            p.H[cc] = fld[1] + cc * cs;
            p.En[cc] = fld[2] + cc * cs;
            p.Hn[cc] = fld[3] + cc * cs;
            for (int t = 0; t < 2; ++t) {
                const int a = (cc + 1 + t) % 3;
                const size_t m = (size_t)(c->ncell / n[a]) * p.W[a];
                p.psiE[cc][t] = talloc(m);
                p.psiH[cc][t] = talloc(m);
                p.psiHn[cc][t] = talloc(m);
            }
        }
        if (fused) {
            for (int par = 0; par < 2; ++par) {
                encode_map(&maps[par].e, par ? fld[2] : fld[0], kSYE);
                encode_map(&maps[par].h, par ? fld[3] : fld[1], kSYH);
            }
            CK(fdtd::prepare_step<T>());
        }
        // CPML tables {1/kappa, b, c, 0} per slab index
        for (int a = 0; a < 3; ++a) {
            const int W = p.W[a];
            std::vector<T> te(4 * std::max(W, 1), T(0)), th(4 * std::max(W, 1), T(0));
            for (int s = 0; s < W; ++s) {
                const int l = s < p.cpl[a] ? s : n[a] - p.cph[a] + (s - p.cpl[a]);
                double ki, b, cc2;
                pml_point(d, c->dt, p.cpl[a], p.cph[a], n[a], (double)l, &ki, &b, &cc2);
                te[4 * s] = (T)ki;
                te[4 * s + 1] = (T)b;
                te[4 * s + 2] = (T)cc2;
                pml_point(d, c->dt, p.cpl[a], p.cph[a], n[a], l + 0.5, &ki, &b, &cc2);
                th[4 * s] = (T)ki;
                th[4 * s + 1] = (T)b;
                th[4 * s + 2] = (T)cc2;
            }
            T* de = talloc(te.size());
            T* dh = talloc(th.size());
            CK(cudaMemcpyAsync(de, te.data(), te.size() * sizeof(T), cudaMemcpyHostToDevice, c->work));
            CK(cudaMemcpyAsync(dh, th.data(), th.size() * sizeof(T), cudaMemcpyHostToDevice, c->work));
            p.pmlE[a] = de;
            p.pmlH[a] = dh;
        }
        p.inv_dx = (T)(1.0 / d.dx);
        p.ch = (T)(c->dt / kMu0);
        const bool per_sample = c->d.density_layout == 1;
        rho = talloc((per_sample ? 3 : 1) * c->nd);
        p.rho = rho;
        for (int cc = 0; cc < 3; ++cc) {
            p.rhoc[cc] = per_sample ? rho + cc * c->nd : rho;
            std::memcpy(p.mb[cc], c->dbu, sizeof p.mb[cc]);
            if (per_sample && c->nd)
                for (int a = 0; a < 3; ++a)
                    if (a != cc) p.mb[cc][2 * a + 1] += 1;
        }
        poles = (PoleTable<T>*)c->alloc(sizeof(PoleTable<T>));
        CK(cudaMemsetAsync(poles, 0, sizeof(PoleTable<T>), c->work));
        p.poles = poles;
        int pmax = 0;
        for (int k = 0; k < 3; ++k) {
            ptot[k] = p_total[k];
            pmax = std::max(pmax, ptot[k]);
            p.Q[k] = (cpx<T>*)c->alloc(c->nd * std::max(ptot[k], 1) * sizeof(cpx<T>));
        }
        bucket = fdtd::pole_bucket(pmax);
        for (int m = 0; m < 2; ++m) dft[m] = (double2*)c->alloc(c->nd * 3 * d.n_freq * sizeof(double2));
        // phase table (cos, sin)(w_f n dt), n = 0..M, evaluated in FP64 and stored in T
        {
            std::vector<V2> ph((size_t)(d.n_steps + 1) * d.n_freq);
            for (int s = 0; s <= d.n_steps; ++s)
                for (int f = 0; f < d.n_freq; ++f) {
                    const double arg = 2.0 * kPi * c->freqs[f] * c->dt * (double)s;
                    V2 v;
                    v.x = (T)std::cos(arg);
                    v.y = (T)std::sin(arg);
                    ph[(size_t)s * d.n_freq + f] = v;
                }
            phase = (V2*)c->alloc(ph.size() * sizeof(V2));
            CK(cudaMemcpyAsync(phase, ph.data(), ph.size() * sizeof(V2), cudaMemcpyHostToDevice, c->work));
        }
        p.K = fdtd::kMaxSnap;
        snap = talloc((size_t)fdtd::kMaxSnap * 3 * c->nd);
        p.snap = snap;
        staging = c->alloc(std::max<size_t>(std::max(c->nd, c->nvar), 1) * sizeof(double));
        for (int m = 0; m < 2; ++m) {
            dp[m].nd = (long long)c->nd;
            dp[m].nf = d.n_freq;
            dp[m].K = fdtd::kMaxSnap;
            dp[m].snap = snap;
            dp[m].dft = dft[m];
            dp[m].ph = phase;
        }
        ctl = (int*)c->alloc(4 * sizeof(int));
        CK(cudaMemsetAsync(ctl, 0, 4 * sizeof(int), c->work));
        p.ctl = ctl;
        for (int m = 0; m < 2; ++m) dp[m].ctl = ctl;
        shell.pair = shell_pairable(p) ? 1 : 0;
        p.nblocks_s = fdtd::shell_blocks(shell);
        p.edz = 1;
        p.ed_pair = design_pairable() ? 1 : 0;
        p.nblocks_d = c->nd ? fdtd::design_blocks(p.ed_pair ? c->dn[0] / 2 : c->dn[0], c->dn[1], c->dn[2], p.edz,
                                                  FDTD_ED_FLAT && !p.ed_pair)
                            : 0;
        p.nblocks_e = p.nblocks_s + p.nblocks_d;
        p.blowup = (T)1e30;
        p.n_steps = d.n_steps;
        p.tfsf_i0 = -1;
        p.nb = 0;
        std::fill(p.sb, p.sb + 6, 0);
        einc = talloc(d.n_steps);
        hinc = talloc(d.n_steps);
        CK(cudaMemsetAsync(einc, 0, d.n_steps * sizeof(T), c->work));
        CK(cudaMemsetAsync(hinc, 0, d.n_steps * sizeof(T), c->work));
        p.einc = einc;
        p.hinc = hinc;
        // point-source tables: forward (1 basis, 1 voxel box), adjoint (2F bases, gap box)
        src_wave[0] = talloc(d.n_steps);
        src_r[0] = talloc(3);
        src_wave[1] = talloc((size_t)d.n_steps * 2 * d.n_freq);
        src_r[1] = talloc(std::max<size_t>(c->ngap * 3 * 2 * d.n_freq, 1));
        gapbuf = (double2*)c->alloc(std::max<size_t>(c->ngap * 3 * d.n_freq, 1) * sizeof(double2));
        const size_t nout = std::max(c->nd, c->nvar);
        grad = (double*)c->alloc(std::max<size_t>(nout, 1) * sizeof(double));
        const size_t nblk = (nout + fdtd::kReduceThreads - 1) / fdtd::kReduceThreads;
        partial = (double*)c->alloc((nblk + 1) * sizeof(double));
        counter = (unsigned*)c->alloc(sizeof(unsigned));
        CK(cudaMemsetAsync(counter, 0, sizeof(unsigned), c->work));
        AB = (double2*)c->alloc(3 * d.n_freq * 2 * sizeof(double2));
        pf = base;
        pa = base;
        build_forward_source();
    }

    void build_forward_source()
    {
        const fdtd_grid_desc& d = c->d;
        if (d.src_kind == 0) {
            std::vector<T> w(d.n_steps), r(3, T(0));
            for (int s = 0; s < d.n_steps; ++s) w[s] = (T)src_pulse(d, c->dt, (s + 0.5) * c->dt);
            r[d.src_comp] = (T)(d.src_amp * kEps0 / c->dt);
            CK(cudaMemcpyAsync(src_wave[0], w.data(), w.size() * sizeof(T), cudaMemcpyHostToDevice, c->work));
            CK(cudaMemcpyAsync(src_r[0], r.data(), 3 * sizeof(T), cudaMemcpyHostToDevice, c->work));
            pf.nb = 1;
            pf.src_r = src_r[0];
            pf.src_wave = src_wave[0];
            const int sb[6] = {d.src_pos[0], d.src_pos[0] + 1, d.src_pos[1], d.src_pos[1] + 1, d.src_pos[2], d.src_pos[2] + 1};
            std::memcpy(pf.sb, sb, sizeof sb);
            pf.tfsf_i0 = -1;
        } else {
            pf.nb = 0;
            pf.tfsf_i0 = d.src_pos[0];
        }
    }

    // Incident plane wave of the one-sided TF/SF source: a 1-D Yee line along x with the grid's
    // dx and dt in the background's z-component medium, hard-driven at its first node; node 2
    // maps onto the first total-field plane.  Long enough that its far end never echoes back.
    void build_incident(const Material& bg)
    {
        const fdtd_grid_desc& d = c->d;
        if (d.src_kind != 1) return;
        const int M = d.n_steps, off = 2;
        const int L = off + (int)std::ceil(0.6 * M) + 16;
        std::vector<double> e(L, 0.0), h(L, 0.0);
        std::vector<T> ei(M), hi(M);
        const double dt = c->dt, dx = d.dx;
        const double Dp = kEps0 * bg.eps[2] / dt + 0.5 * bg.sig[2];
        const double Dm = kEps0 * bg.eps[2] / dt - 0.5 * bg.sig[2];
        const double chx = dt / (kMu0 * dx);
        e[0] = d.src_amp * src_pulse(d, c->dt, 0.0);
        for (int s = 0; s < M; ++s) {
            ei[s] = (T)e[off];
            for (int m = 0; m + 1 < L; ++m) h[m] += chx * (e[m + 1] - e[m]);
            h[L - 1] += chx * (0.0 - e[L - 1]);
            hi[s] = (T)h[off - 1];
            for (int m = 1; m < L; ++m) e[m] = (Dm * e[m] + (h[m] - h[m - 1]) / dx) / Dp;
            e[0] = d.src_amp * src_pulse(d, c->dt, (s + 1) * dt);
        }
        CK(cudaMemcpyAsync(einc, ei.data(), M * sizeof(T), cudaMemcpyHostToDevice, c->work));
        CK(cudaMemcpyAsync(hinc, hi.data(), M * sizeof(T), cudaMemcpyHostToDevice, c->work));
    }

    Material mat_m1, mat_m2;        // the design materials (paper-mode gradient constants)
    double mat_gamma = 0.0;

    void set_materials(const Material& bg, const Material& m1, const Material& m2, double gamma)
    {
        mat_m1 = m1;
        mat_m2 = m2;
        mat_gamma = gamma;
        pm_have_fwd = false;
        const double dt = c->dt;
        PoleTable<T> tab;
        std::memset(&tab, 0, sizeof tab);
        std::vector<double2> ab(3 * c->d.n_freq * 2);
        for (int k = 0; k < 3; ++k) {
            const int P1 = (int)m1.poles[k].size(), P2 = (int)m2.poles[k].size();
            if (P1 + P2 != ptot[k]) arg_error("pole counts differ from those the handle was created with");
            // background
            {
                const double Dp = kEps0 * bg.eps[k] / dt + 0.5 * bg.sig[k];
                const double Dm = kEps0 * bg.eps[k] / dt - 0.5 * bg.sig[k];
                if (!(Dp > 0.0)) arg_error("background update denominator <= 0");
                base.bg_ca[k] = (T)(Dm / Dp);
                base.bg_cb[k] = (T)(1.0 / Dp);
                base.bg_cbi[k] = (T)(1.0 / (Dp * c->d.dx));
            }
            double D[2], N[2];
            const Material* mm[2] = {&m1, &m2};
            for (int i = 0; i < 2; ++i) {
                double sb = 0.0;
                for (const Pole& q : mm[i]->poles[k]) {
                    const cd am1 = expm1c(q.a * dt);
                    sb += (kEps0 * q.c * am1 / (2.0 * q.a)).real();
                }
                D[i] = kEps0 * mm[i]->eps[k] / dt + 0.5 * mm[i]->sig[k] + 2.0 * sb / dt;
                N[i] = kEps0 * mm[i]->eps[k] / dt - 0.5 * mm[i]->sig[k] - 2.0 * sb / dt;
                if (!(D[i] > 0.0)) arg_error("material update denominator <= 0 (eps_inf too small for these poles)");
            }
            base.D1[k] = (T)D[0];
            base.dD[k] = (T)(D[1] - D[0]);
            base.N1[k] = (T)N[0];
            base.dN[k] = (T)(N[1] - N[0]);
            base.P[k] = P1 + P2;
            base.P1[k] = P1;
            std::vector<cd> alpha(P1 + P2), beta(P1 + P2), am1v(P1 + P2);
            for (int p = 0; p < P1 + P2; ++p) {
                const Pole& q = p < P1 ? m1.poles[k][p] : m2.poles[k][p - P1];
                const cd am1 = expm1c(q.a * dt);
                const cd be = kEps0 * q.c * am1 / (2.0 * q.a);
                am1v[p] = am1;
                alpha[p] = 1.0 + am1;
                beta[p] = be;
                tab.am1[k][p] = cpx<T>{(T)am1.real(), (T)am1.imag()};
                tab.beta[k][p] = cpx<T>{(T)be.real(), (T)be.imag()};
                const cd g = 2.0 / dt * am1;
                tab.g[k][p] = cpx<T>{(T)g.real(), (T)g.imag()};
            }
            // gradient constants: dY/drho = A + (1 - 2 rho) B at each objective frequency
            for (int f = 0; f < c->d.n_freq; ++f) {
                const double wdt = 2.0 * kPi * c->freqs[f] * dt;
                const double s = std::sin(0.5 * wdt);
                const cd zm1(-2.0 * s * s, std::sin(wdt));    // z - 1
                const cd zp1 = zm1 + 2.0;                       // z + 1
                cd poles_sum = 0.0;
                for (int p = 0; p < P1 + P2; ++p) {
                    const cd h = beta[p] * zp1 / (zm1 - am1v[p]) + std::conj(beta[p]) * zp1 / (zm1 - std::conj(am1v[p]));
                    poles_sum += (p < P1) ? -h : h;
                }
                const cd A = (kEps0 * (m2.eps[k] - m1.eps[k]) * zm1 + (m2.sig[k] - m1.sig[k]) * dt * zp1 / 2.0 + zm1 * poles_sum) / dt;
                const cd B = gamma * zp1 / 2.0;
                ab[(k * c->d.n_freq + f) * 2] = make_double2(A.real(), A.imag());
                ab[(k * c->d.n_freq + f) * 2 + 1] = make_double2(B.real(), B.imag());
            }
        }
        if (!(gamma >= 0.0)) arg_error("gamma must be >= 0");
        base.hg = (T)(0.5 * gamma);
        CK(cudaMemcpyAsync(poles, &tab, sizeof tab, cudaMemcpyHostToDevice, c->work));
        htab = tab;
        ab_host = ab;
        CK(cudaMemcpyAsync(AB, ab_host.data(), ab_host.size() * sizeof(double2), cudaMemcpyHostToDevice, c->work));
        build_incident(bg);
        refresh_params();
    }

    // Copy the material part of `base` into the forward / adjoint parameter sets.
    void refresh_params()
    {
        KParams<T> f = base, a = base;
        f.nb = pf.nb;
        f.src_r = pf.src_r;
        f.src_wave = pf.src_wave;
        std::memcpy(f.sb, pf.sb, sizeof f.sb);
        f.tfsf_i0 = pf.tfsf_i0;
        a.nb = pa.nb;
        a.src_r = pa.src_r;
        a.src_wave = pa.src_wave;
        std::memcpy(a.sb, pa.sb, sizeof a.sb);
        a.tfsf_i0 = -1;
        pf = f;
        pa = a;
        drop_graphs();
    }

    size_t cs = 0;                  // component stride of a field block (elements)

    // 4-D (x, y, z, component) tiled map of a field block; box kSX x rows x 1 x 3, zero fill outside.
    void encode_map(CUtensorMap* m, T* base_ptr, int rows)
    {
        const fdtd_grid_desc& d = c->d;
        const cuuint64_t dims[4] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz, 3};
        const cuuint64_t strides[3] = {(cuuint64_t)d.nx * sizeof(T), (cuuint64_t)d.nx * d.ny * sizeof(T),
                                       (cuuint64_t)cs * sizeof(T)};
        const cuuint32_t box[4] = {(cuuint32_t)kSX, (cuuint32_t)rows, 1, 3};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        const CUresult r = tensor_map_encoder()(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                                                4, base_ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) throw Err{FDTD_ERR_CUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r)};
    }

    // Interior box of the fused kernel: kTX x kTY tiles whose cells and one-cell -x/-y halo lie outside
    // the walls and the CPML slabs, x0 a multiple of 4 (16-byte aligned TMA boxes), planes cpml_z_low + 1
    // .. nz - cpml_z_high - 1 (the plane below the first one is outside the slab too), at least one whole
    // tile each way.  Toward the +x and +y slabs the box ends in a partial tile column or row (an even
    // number of x cells; the kernel leaves the cells beyond to the shell) when that tile holds at least
    // FDTD_PARTIAL_MIN_X columns / FDTD_PARTIAL_MIN_Y rows: a partial tile costs a whole tile's work
    // (FDTD_PARTIAL_TILES 0: whole tiles only).  Needs x rows of a multiple of 16 bytes and the tensor-map
    // encoder.  The rest of the grid is the shell: at most six boxes.
#ifndef FDTD_STEP_MINBLK
#define FDTD_STEP_MINBLK (2 * 152)
#endif
#ifndef FDTD_PARTIAL_TILES
#define FDTD_PARTIAL_TILES 1
#endif
#ifndef FDTD_PARTIAL_MIN_X
#define FDTD_PARTIAL_MIN_X 24   // x cells a partial last tile column must hold (of kTX)
#endif
#ifndef FDTD_PARTIAL_MIN_Y
#define FDTD_PARTIAL_MIN_Y 12   // rows a partial last tile row must hold (of kTY)
#endif
    void split_grid(KParams<T>& p)
    {
        const fdtd_grid_desc& d = c->d;
        const int X0 = (std::max(p.cpl[0] + 1, 1) + 3) / 4 * 4, Y0 = std::max(p.cpl[1] + 1, 1), Z0 = p.cpl[2] + 1;
        const int wx = d.nx - p.cph[0] - X0, wy = d.ny - p.cph[1] - Y0;   // widths up to the +x / +y slabs
        const int Z1 = d.nz - p.cph[2];
        fused = ((size_t)d.nx * sizeof(T)) % 16 == 0 && wx >= fdtd::kTX && wy >= fdtd::kTY && Z1 > Z0 &&
                tensor_map_encoder() != nullptr;
        const int rx = (wx & ~1) % fdtd::kTX, ry = wy % fdtd::kTY;   // cells of a partial last tile
        const int X1 = X0 + wx / fdtd::kTX * fdtd::kTX + (FDTD_PARTIAL_TILES && rx >= FDTD_PARTIAL_MIN_X ? rx : 0);
        const int Y1 = Y0 + wy / fdtd::kTY * fdtd::kTY + (FDTD_PARTIAL_TILES && ry >= FDTD_PARTIAL_MIN_Y ? ry : 0);
        const int ntx = (X1 - X0 + fdtd::kTX - 1) / fdtd::kTX, nty = (Y1 - Y0 + fdtd::kTY - 1) / fdtd::kTY;
        const int ib[6] = {X0, X1, Y0, Y1, Z0, Z1};
        std::fill(p.ib, p.ib + 6, 0);
        if (fused) std::copy(ib, ib + 6, p.ib);
        // z planes per block: kKC, halved while the launch has fewer than FDTD_STEP_MINBLK blocks
        p.kc = fdtd::kKC;
        if (fused)
            while (p.kc > 2 && (unsigned)ntx * nty * ((Z1 - Z0 + p.kc - 1) / p.kc) < FDTD_STEP_MINBLK) p.kc /= 2;
        shell = fdtd::ShellBoxes{};
        auto add = [&](int x0, int x1, int y0, int y1, int z0, int z1) {
            if (x0 >= x1 || y0 >= y1 || z0 >= z1) return;
            int* b = shell.b[shell.n++];
            b[0] = x0; b[1] = x1; b[2] = y0; b[3] = y1; b[4] = z0; b[5] = z1;
        };
        if (!fused) {
            add(0, d.nx, 0, d.ny, 0, d.nz);
        } else {
            add(0, d.nx, 0, d.ny, 0, ib[4]);                      // below and above the interior planes
            add(0, d.nx, 0, d.ny, ib[5], d.nz);
            add(0, d.nx, 0, ib[2], ib[4], ib[5]);                 // in front of and behind it in y
            add(0, d.nx, ib[3], d.ny, ib[4], ib[5]);
            add(0, ib[0], ib[2], ib[3], ib[4], ib[5]);            // left and right of it in x
            add(ib[1], d.nx, ib[2], ib[3], ib[4], ib[5]);
        }
    }

    // The paired shell kernels (FP32) need the x boundaries of the grid, of the CPML slabs and of the
    // shell boxes even (the two cells of a pair on the same side of each); the working box's x bounds,
    // the TF/SF plane and point sources may fall between the cells of a pair.
    bool shell_pairable(const KParams<T>& p) const
    {
        if (sizeof(T) != 4 || p.nx % 2 || p.cpl[0] % 2 || p.cph[0] % 2) return false;
        for (int q = 0; q < shell.n; ++q)
            if (shell.b[q][0] % 2 || shell.b[q][1] % 2) return false;
        return true;
    }

    // The paired design-E kernel (FP32) needs nx and the working box's x origin and extent even (a pair's
    // samples adjacent and 8-byte aligned in the fields, densities, snapshots and pole currents), and up
    // to 8 poles a component (more would spill the pair's pole currents).
    // FDTD_ED_PAIR 0 (build knob) keeps the one-sample kernel.
    bool design_pairable() const
    {
#if defined(FDTD_ED_PAIR) && !FDTD_ED_PAIR
        return false;
#else
        const fdtd_grid_desc& d = c->d;
        return sizeof(T) == 4 && c->nd && bucket <= 8 && d.nx % 2 == 0 && d.design_box[0] % 2 == 0 &&
               c->dn[0] % 2 == 0;
#endif
    }

    // Background part of one step: H of the shell and the fused interior (both read only the old
    // buffers), then E of the shell (reads the new H of its neighbours).  concurrent: the shell H runs
    // on the side stream next to the interior kernel (graph capture); else all three in order.
    cudaError_t launch_background(const KParams<T>& q, int parity, bool concurrent, const StepMaps* mp = nullptr)
    {
        if (!mp) mp = maps;
        cudaError_t e = cudaSuccess;
        if (concurrent && fused) {
            e = cudaEventRecord(c->fork, c->work);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->fork, 0);
            if (e == cudaSuccess) e = fdtd::launch_shell<T>(q, shell, false, c->side);
            if (e == cudaSuccess) e = fdtd::launch_step<T>(q, mp[parity & 1], c->work);
            if (e == cudaSuccess) e = cudaEventRecord(c->join, c->side);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(c->work, c->join, 0);
        } else {
            e = fdtd::launch_shell<T>(q, shell, false, c->work);
            if (e == cudaSuccess && fused) e = fdtd::launch_step<T>(q, mp[parity & 1], c->work);
        }
        return e == cudaSuccess ? fdtd::launch_shell<T>(q, shell, true, c->work) : e;
    }

    // One whole time step: the H phase (shell H next to the interior kernel when concurrent), then
    // the E phase, whose shell E and design E kernels write disjoint cells and run side by side when
    // concurrent (the last block of the two advances the step counter).
    cudaError_t launch_one_step(const KParams<T>& q, int parity, bool concurrent, const StepMaps* mp = nullptr)
    {
        if (!concurrent || c->nd == 0) {
            cudaError_t e = launch_background(q, parity, concurrent, mp);
            return e == cudaSuccess ? fdtd::launch_e_design<T>(q, htab, bucket, c->work) : e;
        }
        if (!mp) mp = maps;
        cudaError_t e = cudaEventRecord(c->fork, c->work);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->fork, 0);
        if (e == cudaSuccess) e = fdtd::launch_shell<T>(q, shell, false, c->side);
        if (e == cudaSuccess && fused) e = fdtd::launch_step<T>(q, mp[parity & 1], c->work);
        if (e == cudaSuccess) e = cudaEventRecord(c->join, c->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->work, c->join, 0);
        if (e == cudaSuccess) e = cudaEventRecord(c->fork, c->work);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->fork, 0);
        if (e == cudaSuccess) e = fdtd::launch_shell<T>(q, shell, true, c->side);
        if (e == cudaSuccess) e = fdtd::launch_e_design<T>(q, htab, bucket, c->work);
        if (e == cudaSuccess) e = cudaEventRecord(c->join, c->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->work, c->join, 0);
        return e;
    }

    // Parameters of a step with the given parity: odd steps read the second buffer of each pair.
    KParams<T> par(const KParams<T>& p, int parity) const
    {
        if (!(parity & 1)) return p;
        KParams<T> q = p;
        for (int cc = 0; cc < 3; ++cc) {
            std::swap(q.E[cc], q.En[cc]);
            std::swap(q.H[cc], q.Hn[cc]);
            for (int t = 0; t < 2; ++t) std::swap(q.psiH[cc][t], q.psiHn[cc][t]);
        }
        return q;
    }

    // ---- paper mode ----------------------------------------------------------------------------
    // The time-domain energy objective of Eq. (Objective_analyitically_enhancement) and its gradient by
    // Eq. (Gradient_FDTD), with checkpoint-recompute instead of the paper's full histories: the forward
    // run stores its whole state every C steps; the gradient pass takes the segments last first,
    // recomputes each one recording the design-box E and the pole term, advances the adjoint system (a
    // second state set, driven by the time-reversed gap field) over the mirrored steps recording its
    // design-box E, and accumulates the segment's terms per voxel.  Reading of the half-step alignment:
    // the adjoint drive is eps0 E^{M-m-1} at adjoint step m, and the adjoint levels m, m-1 stand for the
    // paper's m+1/2, m-1/2.
    struct StateSet {
        T* fld[4] = {nullptr, nullptr, nullptr, nullptr};   // E, H, E', H' blocks (3 * cs each)
        T* psiE[3][2] = {};
        T* psiH[3][2] = {};
        T* psiHn[3][2] = {};
        cpx<T>* Q[3] = {};
        int* ctl = nullptr;
    };
    bool pm_ready = false;
    int pm_C = 0, pm_nseg = 0;
    StateSet pm_b;                                   // adjoint state
    StepMaps pm_maps[2]{};
    KParams<T> pm_fwd{}, pm_rec{}, pm_adj{};         // forward pass, recompute pass, adjoint pass
    unsigned char* pm_ckpt = nullptr;                // pm_nseg slabs of pm_ckpt_bytes
    size_t pm_ckpt_bytes = 0;
    T *pm_he = nullptr, *pm_ha = nullptr, *pm_hq = nullptr, *pm_gh = nullptr, *pm_drive = nullptr;
    double *pm_td = nullptr, *pm_gsum = nullptr;
    bool pm_have_fwd = false;

    size_t psi_elems(int cc, int t) const
    {
        const int n[3] = {c->d.nx, c->d.ny, c->d.nz};
        const int a = (cc + 1 + t) % 3;
        return (size_t)(c->ncell / n[a]) * base.W[a];
    }

    // The state words of a step-parity view: E^n, H^{n-1/2}, psi_E, psi_H^{n-1/2}, Q.
    std::vector<std::pair<void*, size_t>> state_regions(const KParams<T>& q) const
    {
        std::vector<std::pair<void*, size_t>> r;
        r.push_back({q.E[0], 3 * cs * sizeof(T)});
        r.push_back({q.H[0], 3 * cs * sizeof(T)});
        for (int cc = 0; cc < 3; ++cc)
            for (int t = 0; t < 2; ++t) {
                const size_t m = psi_elems(cc, t);
                if (m) {
                    r.push_back({q.psiE[cc][t], m * sizeof(T)});
                    r.push_back({q.psiH[cc][t], m * sizeof(T)});
                }
            }
        for (int cc = 0; cc < 3; ++cc)
            if (ptot[cc] && c->nd) r.push_back({q.Q[cc], c->nd * ptot[cc] * sizeof(cpx<T>)});
        return r;
    }

    void copy_state(const KParams<T>& q, unsigned char* slab, bool save)
    {
        size_t off = 0;
        for (auto& reg : state_regions(q)) {
            if (save) CK(cudaMemcpyAsync(slab + off, reg.first, reg.second, cudaMemcpyDeviceToDevice, c->work));
            else CK(cudaMemcpyAsync(reg.first, slab + off, reg.second, cudaMemcpyDeviceToDevice, c->work));
            off += (reg.second + 255) / 256 * 256;
        }
    }

    void pm_alloc(int C)
    {
        const fdtd_grid_desc& d = c->d;
        const int M = d.n_steps;
        if (c->nd == 0 || c->ngap == 0) arg_error("paper mode needs a design box with a gap");
        if (d.density_layout != 0) arg_error("paper mode takes one density per voxel (density_layout 0)");
        if (!pm_b.fld[0]) {                      // adjoint state set, allocated once
            for (int f = 0; f < 4; ++f) pm_b.fld[f] = talloc(3 * cs);
            for (int cc = 0; cc < 3; ++cc)
                for (int t = 0; t < 2; ++t) {
                    const size_t m = psi_elems(cc, t);
                    pm_b.psiE[cc][t] = talloc(m);
                    pm_b.psiH[cc][t] = talloc(m);
                    pm_b.psiHn[cc][t] = talloc(m);
                }
            for (int cc = 0; cc < 3; ++cc)
                pm_b.Q[cc] = (cpx<T>*)c->alloc(c->nd * std::max(ptot[cc], 1) * sizeof(cpx<T>));
            pm_b.ctl = (int*)c->alloc(4 * sizeof(int));
            if (fused)
                for (int par = 0; par < 2; ++par) {
                    encode_map(&pm_maps[par].e, par ? pm_b.fld[2] : pm_b.fld[0], kSYE);
                    encode_map(&pm_maps[par].h, par ? pm_b.fld[3] : pm_b.fld[1], kSYH);
                }
            const size_t ns = 3 * c->ngap;
            pm_gh = talloc((size_t)M * ns);
            pm_drive = talloc((size_t)M * ns);
            pm_td = (double*)c->alloc(ns * sizeof(double));
            pm_gsum = (double*)c->alloc(c->nd * sizeof(double));
        }
        pm_ckpt_bytes = 0;
        for (auto& reg : state_regions(base)) pm_ckpt_bytes += (reg.second + 255) / 256 * 256;
        const size_t step_hist = 3 * 3 * c->nd * sizeof(T);      // forward E, pole term, adjoint E per step
        if (C <= 0) C = std::max(1, (int)std::lround(std::sqrt((double)M * pm_ckpt_bytes / step_hist)));
        C = std::min(C, M);
        if (pm_ready && C == pm_C) return;
        pm_C = C;
        pm_nseg = (M + C - 1) / C;
        pm_ckpt = (unsigned char*)c->alloc((size_t)pm_nseg * pm_ckpt_bytes);
        pm_he = talloc((size_t)(C + 1) * 3 * c->nd);
        pm_ha = talloc((size_t)(C + 1) * 3 * c->nd);
        pm_hq = talloc((size_t)C * 3 * c->nd);
        pm_ready = true;
    }

    // Step parameters of the three passes, from the current materials and sources.
    void pm_params()
    {
        const int C = pm_C;
        // forward pass: the objective's gap energy and the gap field history (snapshots to scratch)
        pm_fwd = pf;
        pm_fwd.td_acc = pm_td;
        pm_fwd.gap_hist = pm_gh;
        pm_fwd.nsamp = (int)(3 * c->ngap);
        pm_fwd.snap = pm_he;
        pm_fwd.K = C;
        pm_fwd.snap0 = 0;
        // recompute pass: design-box E^{n+1} into slots 1.., the pole term into pm_hq
        pm_rec = pf;
        pm_rec.snap = pm_he + 3 * c->nd;
        pm_rec.hist_dq = pm_hq;
        pm_rec.K = C;
        // adjoint pass: second state set, direct drive table at the gap samples
        pm_adj = base;
        for (int cc = 0; cc < 3; ++cc) {
            pm_adj.E[cc] = pm_b.fld[0] + cc * cs;
            pm_adj.H[cc] = pm_b.fld[1] + cc * cs;
            pm_adj.En[cc] = pm_b.fld[2] + cc * cs;
            pm_adj.Hn[cc] = pm_b.fld[3] + cc * cs;
            for (int t = 0; t < 2; ++t) {
                pm_adj.psiE[cc][t] = pm_b.psiE[cc][t];
                pm_adj.psiH[cc][t] = pm_b.psiH[cc][t];
                pm_adj.psiHn[cc][t] = pm_b.psiHn[cc][t];
            }
            pm_adj.Q[cc] = pm_b.Q[cc];
        }
        pm_adj.ctl = pm_b.ctl;
        pm_adj.nb = 1;
        pm_adj.src_direct = 1;
        pm_adj.nsamp = (int)(3 * c->ngap);
        pm_adj.src_wave = pm_drive;
        std::memcpy(pm_adj.sb, base.gb, sizeof pm_adj.sb);
        pm_adj.tfsf_i0 = -1;
        pm_adj.snap = pm_ha + 3 * c->nd;
        pm_adj.K = C;
    }

    void pm_steps(const KParams<T>& p, const StepMaps* mp, int n_from, int n_to)
    {
        for (int s = n_from; s < n_to; ++s) {
            const KParams<T> q = par(p, s);
            CK(launch_one_step(q, s, true, mp));   // both phases on two streams, as in the captured graphs
        }
        c->tim.launches += (long long)(n_to - n_from) * (fused ? 4 : 3);
    }

    void pm_check(const int* ctl_dev, int expect)
    {
        int h[4];
        CK(cudaMemcpyAsync(h, ctl_dev, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->work));
        CK(cudaStreamSynchronize(c->work));
        if (h[2] & 4) {
            c->dead = true;
            throw Err{FDTD_ERR_TIMEOUT, "a wait of the step kernel gave up after its time limit"};
        }
        if (h[2] & 1) {
            c->dead = true;
            throw Err{FDTD_ERR_UNSTABLE, "non-finite or exploding field during the run"};
        }
        if (h[0] != expect) throw Err{FDTD_ERR_CUDA, "device step counter " + std::to_string(h[0]) + " != " + std::to_string(expect)};
    }

    double paper_forward(int C)
    {
        const int M = c->d.n_steps;
        pm_alloc(C);
        pm_params();
        reset_state(0);
        CK(cudaMemsetAsync(pm_td, 0, 3 * c->ngap * sizeof(double), c->work));
        for (int seg = 0; seg < pm_nseg; ++seg) {
            const int n0 = seg * pm_C, n1 = std::min(M, n0 + pm_C);
            copy_state(par(pm_fwd, n0), pm_ckpt + (size_t)seg * pm_ckpt_bytes, true);
            pm_steps(pm_fwd, maps, n0, n1);
            if (c->cancel.load()) throw Err{FDTD_ERR_CANCELLED, "cancelled"};
        }
        pm_check(ctl, M);
        std::vector<double> td(3 * c->ngap);
        CK(cudaMemcpyAsync(td.data(), pm_td, td.size() * sizeof(double), cudaMemcpyDeviceToHost, c->work));
        CK(cudaStreamSynchronize(c->work));
        double s = 0.0;
        for (double v : td) s += v;
        const double dV = c->d.dx * c->d.dx * c->d.dx;
        pm_have_fwd = true;
        return 0.5 * kEps0 * dV * c->dt * s;
    }

    void paper_gradient(int single, void* out, int dtype, int on_device)
    {
        if (!pm_have_fwd) throw Err{FDTD_ERR_STATE, "paper gradient before paper forward"};
        pm_params();
        const fdtd_grid_desc& d = c->d;
        const int M = d.n_steps;
        const size_t ns = 3 * c->ngap;
        CK(fdtd::launch_paper_drive<T>(pm_gh, pm_drive, M, (int)ns, kEps0, c->work));
        // adjoint state to zero
        for (int f = 0; f < 4; ++f) CK(cudaMemsetAsync(pm_b.fld[f], 0, 3 * cs * sizeof(T), c->work));
        for (int cc = 0; cc < 3; ++cc)
            for (int t = 0; t < 2; ++t) {
                const size_t m = psi_elems(cc, t);
                if (!m) continue;
                CK(cudaMemsetAsync(pm_b.psiE[cc][t], 0, m * sizeof(T), c->work));
                CK(cudaMemsetAsync(pm_b.psiH[cc][t], 0, m * sizeof(T), c->work));
                CK(cudaMemsetAsync(pm_b.psiHn[cc][t], 0, m * sizeof(T), c->work));
            }
        for (int cc = 0; cc < 3; ++cc)
            if (ptot[cc]) CK(cudaMemsetAsync(pm_b.Q[cc], 0, c->nd * ptot[cc] * sizeof(cpx<T>), c->work));
        CK(cudaMemsetAsync(pm_b.ctl, 0, 4 * sizeof(int), c->work));
        CK(cudaMemsetAsync(pm_gsum, 0, c->nd * sizeof(double), c->work));
        fdtd::PParams<T> g{};
        g.nd = (long long)c->nd;
        g.dnx = base.dnx;
        g.dny = base.dny;
        std::memcpy(g.db, base.db, sizeof g.db);
        std::memcpy(g.gb, base.gb, sizeof g.gb);
        g.he = pm_he;
        g.ha = pm_ha;
        g.hq = pm_hq;
        g.rho = rho;
        g.gsum = pm_gsum;
        g.single = single ? 1 : 0;
        for (int k = 0; k < 3; ++k) {
            g.deps[k] = mat_m2.eps[k] - mat_m1.eps[k];
            g.dsig[k] = mat_m2.sig[k] - mat_m1.sig[k];
        }
        g.gamma = mat_gamma;
        g.eps0 = kEps0;
        g.dt = c->dt;
        for (int seg = pm_nseg - 1; seg >= 0; --seg) {
            const int n0 = seg * pm_C, n1 = std::min(M, n0 + pm_C), len = n1 - n0, a0 = M - n1;
            // forward recompute of the segment from its checkpoint
            KParams<T> pr = pm_rec;
            pr.snap0 = n0;
            copy_state(par(pr, n0), pm_ckpt + (size_t)seg * pm_ckpt_bytes, false);
            CK(cudaMemcpyAsync(ctl, &n0, sizeof(int), cudaMemcpyHostToDevice, c->work));
            CK(fdtd::launch_gather_design_e<T>(par(pr, n0), pm_he, c->work));
            pm_steps(pr, maps, n0, n1);
            // adjoint over the mirrored steps a0 .. a0 + len
            KParams<T> pa2 = pm_adj;
            pa2.snap0 = a0;
            CK(fdtd::launch_gather_design_e<T>(par(pa2, a0), pm_ha, c->work));
            pm_steps(pa2, pm_maps, a0, a0 + len);
            g.len = len;
            CK(fdtd::launch_paper_grad<T>(g, c->work));
            c->tim.launches += 3;
            CK(cudaStreamSynchronize(c->work));      // n0 above is a host stack value read by the copy
            if (c->cancel.load()) throw Err{FDTD_ERR_CANCELLED, "cancelled"};
        }
        pm_check(pm_b.ctl, M);
        std::vector<double> gs(c->nd);
        CK(cudaMemcpyAsync(gs.data(), pm_gsum, c->nd * sizeof(double), cudaMemcpyDeviceToHost, c->work));
        CK(cudaStreamSynchronize(c->work));
        const double dV = d.dx * d.dx * d.dx;
        for (double& v : gs) v *= dV;
        if (!out) return;
        const cudaMemcpyKind kind = on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
        if (dtype == 1) {
            CK(cudaMemcpyAsync(out, gs.data(), c->nd * sizeof(double), kind, c->work));
            CK(cudaStreamSynchronize(c->work));
        } else {
            std::vector<float> gf(gs.begin(), gs.end());
            CK(cudaMemcpyAsync(out, gf.data(), c->nd * sizeof(float), kind, c->work));
            CK(cudaStreamSynchronize(c->work));
        }
    }

    // Buffers that hold the state after a run of M steps.
    T* cur_field(int which) const
    {
        const bool odd = c->d.n_steps & 1;
        if (which < 3) return odd ? base.En[which] : base.E[which];
        return odd ? base.Hn[which - 3] : base.H[which - 3];
    }

    void drop_graphs()
    {
        for (auto& g : graph)
            for (auto& x : g)
                if (x) {
                    cudaGraphExecDestroy(x);
                    x = nullptr;
                }
    }

    void set_density(const void* src, int dtype, int on_device)
    {
        pm_have_fwd = false;
        const bool per_sample = c->d.density_layout == 1;
        const size_t n = c->nvar;
        int* flag = ctl + 2;
        CK(cudaMemsetAsync(ctl, 0, 4 * sizeof(int), c->work));
        const void* dsrc = src;
        if (!on_device) {   // host (pageable or pinned) -> staging, checked and converted on the device
            CK(cudaMemcpyAsync(staging, src, n * (dtype == 0 ? 4 : 8), cudaMemcpyHostToDevice, c->work));
            dsrc = staging;
        }
        if (per_sample) {   // compact per-component samples -> the three working-box arrays
            CK(cudaMemsetAsync(rho, 0, 3 * c->nd * sizeof(T), c->work));
            CK(fdtd::launch_rho_scatter<T>(dsrc, dtype, (long long)n, c->voff, c->vdim, c->dn[0], c->dn[1],
                                           (long long)c->nd, rho, flag, c->work));
        } else {
            CK(fdtd::launch_rho_import<T>(dsrc, dtype, (long long)n, rho, flag, c->work));
        }
        c->tim.launches++;
        int hflag[4];
        CK(cudaMemcpyAsync(hflag, ctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->work));
        CK(cudaStreamSynchronize(c->work));
        if (hflag[2] & 2) arg_error("density value out of [0, 1] or non-finite");
    }

    void reset_state(int mode)
    {
        cudaStream_t s = c->work;
        for (int k = 0; k < 3; ++k) {
            CK(cudaMemsetAsync(base.E[k], 0, c->ncell * sizeof(T), s));
            CK(cudaMemsetAsync(base.H[k], 0, c->ncell * sizeof(T), s));
            CK(cudaMemsetAsync(base.En[k], 0, c->ncell * sizeof(T), s));
            CK(cudaMemsetAsync(base.Hn[k], 0, c->ncell * sizeof(T), s));
            for (int t = 0; t < 2; ++t) {
                const int a = (k + 1 + t) % 3;
                const int n[3] = {c->d.nx, c->d.ny, c->d.nz};
                const size_t m = (size_t)(c->ncell / n[a]) * base.W[a];
                if (m) {
                    CK(cudaMemsetAsync(base.psiE[k][t], 0, m * sizeof(T), s));
                    CK(cudaMemsetAsync(base.psiH[k][t], 0, m * sizeof(T), s));
                    CK(cudaMemsetAsync(base.psiHn[k][t], 0, m * sizeof(T), s));
                }
            }
            if (ptot[k] && c->nd) CK(cudaMemsetAsync(base.Q[k], 0, c->nd * ptot[k] * sizeof(cpx<T>), s));
        }
        if (c->nd) CK(cudaMemsetAsync(dft[mode], 0, c->nd * 3 * c->d.n_freq * sizeof(double2), s));
        CK(cudaMemsetAsync(ctl, 0, 4 * sizeof(int), s));
    }

    // The graph of `steps` steps and one DFT launch, built node by node: per step an H phase (shell H
    // kernel, fused interior kernel) and an E phase (shell E kernel, design-E kernel), the two kernels of a
    // phase independent of each other, every kernel of a phase depending on both kernels of the phase
    // before through a programmatic edge.  A phase's blocks are thereby launched while the phase before
    // drains and wait (pdl_wait) until it has completed, instead of being launched after it.  Returns
    // nullptr (and leaves no error state) where the driver refuses such a graph.
    cudaGraphExec_t build_pdl_graph(int mode, int steps)
    {
        const KParams<T>& p = mode ? pa : pf;
        cudaGraph_t g = nullptr;
        if (cudaGraphCreate(&g, 0) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        const bool has_shell = shell.first[shell.n] > 0;   // the fused kernel may cover the whole grid
        cudaGraphEdgeData ed = {};
        ed.type = cudaGraphDependencyTypeProgrammatic;
        ed.from_port = cudaGraphKernelNodePortProgrammatic;
        std::vector<cudaGraphNode_t> prev, cur;
        cudaError_t e = cudaSuccess;
        auto link = [&](cudaGraphNode_t to) {
            for (cudaGraphNode_t from : prev)
                if (e == cudaSuccess) e = cudaGraphAddDependencies(g, &from, &to, &ed, 1);
        };
        auto phase = [&](auto&& add) {
            cur.clear();
            add();
            for (cudaGraphNode_t n : cur) link(n);
            prev = cur;
        };
        for (int st = 0; st < steps && e == cudaSuccess; ++st) {
            const KParams<T> q = par(p, st);
            phase([&] {
                cudaGraphNode_t n = nullptr;
                if (e == cudaSuccess && has_shell && (e = fdtd::graph_shell<T>(g, &n, q, shell, false)) == cudaSuccess)
                    cur.push_back(n);
                if (e == cudaSuccess && fused && (e = fdtd::graph_step<T>(g, &n, q, maps[st & 1])) == cudaSuccess) cur.push_back(n);
            });
            phase([&] {
                cudaGraphNode_t n = nullptr;
                if (e == cudaSuccess && has_shell && (e = fdtd::graph_shell<T>(g, &n, q, shell, true)) == cudaSuccess)
                    cur.push_back(n);
                if (e == cudaSuccess && c->nd && (e = fdtd::graph_e_design<T>(g, &n, q, htab, bucket)) == cudaSuccess)
                    cur.push_back(n);
            });
        }
        if (e == cudaSuccess && c->nd)
            phase([&] {
                cudaGraphNode_t n = nullptr;
                if ((e = fdtd::graph_dft<T>(g, &n, dp[mode], steps)) == cudaSuccess) cur.push_back(n);
            });
        cudaGraphExec_t ex = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return ex;
    }

    void capture(int mode, int which, int steps)
    {
        if (use_pdl) {
            if (cudaGraphExec_t ex = build_pdl_graph(mode, steps)) {
                graph[mode][which] = ex;
                pdl_built = true;
                return;
            }
            use_pdl = false;    // the driver refused the programmatic edges: captured graphs from here on
        }
        const KParams<T>& p = mode ? pa : pf;
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(c->work, cudaStreamCaptureModeThreadLocal));
        cudaError_t err = cudaSuccess;
        for (int s = 0; s < steps && err == cudaSuccess; ++s) {   // graphs start at even steps
            const KParams<T> q = par(p, s);
            err = launch_one_step(q, s, true);
        }
        if (err == cudaSuccess) err = fdtd::launch_dft<T>(dp[mode], steps, c->work);
        cudaError_t e2 = cudaStreamEndCapture(c->work, &g);
        if (err != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            throw Err{FDTD_ERR_CUDA, std::string("graph capture failed: ") + cudaGetErrorString(err != cudaSuccess ? err : e2)};
        }
        cudaGraphExec_t ex = nullptr;
        err = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        CK(err);
        graph[mode][which] = ex;
    }

    void run(int mode)
    {
        const int M = c->d.n_steps;
        reset_state(mode);
        const KParams<T>& p = mode ? pa : pf;
        const int K = std::min(M, kGraphSteps);
        const int nblk = (M + K - 1) / K;
        const int full = M / K, rem = M % K;
        if (!graph[mode][0]) capture(mode, 0, K);
        if (rem && !graph[mode][1]) capture(mode, 1, rem);
        // Profiling samples one 16-step block in kProfEvery: its kernels are launched one by one
        // between CUDA events; every other block is a graph replay, as without profiling.
        int timed_steps = 0, timed_blocks = 0;
        std::vector<int> sampled;
        if (c->prof) {
            const size_t need = 5 * (size_t)M + nblk;
            while (c->ev.size() < need) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e));
                c->ev.push_back(e);
            }
        }
        int s = 0;
        for (int b = 0; b < nblk; ++b) {
            const int cnt = b < full ? K : rem;
            if (c->prof && b % kProfEvery == 0) {
                sampled.push_back(b);
                for (int q = 0; q < cnt; ++q, ++s) {
                    const KParams<T> pp = par(p, s);
                    cudaEvent_t* e = &c->ev[5 * (size_t)s];
                    CK(cudaEventRecord(e[0], c->work));
                    CK(fdtd::launch_shell<T>(pp, shell, false, c->work));
                    CK(cudaEventRecord(e[1], c->work));
                    if (fused) CK(fdtd::launch_step<T>(pp, maps[s & 1], c->work));
                    CK(cudaEventRecord(e[2], c->work));
                    CK(fdtd::launch_shell<T>(pp, shell, true, c->work));
                    CK(cudaEventRecord(e[3], c->work));
                    CK(fdtd::launch_e_design<T>(pp, htab, bucket, c->work));
                    CK(cudaEventRecord(e[4], c->work));
                }
                CK(fdtd::launch_dft<T>(dp[mode], cnt, c->work));
                CK(cudaEventRecord(c->ev[5 * (size_t)M + b], c->work));
            } else {
                CK(cudaGraphLaunch(graph[mode][b < full ? 0 : 1], c->work));
                s += cnt;
            }
            if ((s % kChunkSteps) < K && c->cancel.load()) throw Err{FDTD_ERR_CANCELLED, "cancelled"};
        }
        if (c->prof) {
            CK(cudaStreamSynchronize(c->work));
            for (int b : sampled) {
                const int first = b * K, cnt = std::min(K, M - b * K);
                for (int q = first; q < first + cnt; ++q) {
                    float t[4] = {0, 0, 0, 0};
                    for (int u = 0; u < 4; ++u) CK(cudaEventElapsedTime(&t[u], c->ev[5 * (size_t)q + u], c->ev[5 * (size_t)q + u + 1]));
                    c->tim.shell_h_ms += t[0];
                    c->tim.step_ms += t[1];
                    c->tim.shell_e_ms += t[2];
                    c->tim.ed_ms += t[3];
                }
                float w = 0;
                CK(cudaEventElapsedTime(&w, c->ev[5 * (size_t)(first + cnt - 1) + 4], c->ev[5 * (size_t)M + b]));
                c->tim.dft_ms += w;
                timed_steps += cnt;
                timed_blocks += 1;
            }
        }
        c->tim.shell_h_launches += timed_steps;    // launches that were timed (profiling samples)
        c->tim.shell_e_launches += timed_steps;
        if (fused) c->tim.step_launches += timed_steps;
        if (c->nd) c->tim.ed_launches += timed_steps;
        if (c->nd) {
            c->tim.dft_launches += timed_blocks;
            c->tim.launches += nblk;
        }
        c->tim.launches += ((fused ? 3LL : 2LL) + (c->nd ? 1LL : 0LL)) * M;  // every kernel this run launched
        c->tim.fused_step = fused ? 1 : 0;
        int hctl[4];
        CK(cudaMemcpyAsync(hctl, ctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->work));
        CK(cudaStreamSynchronize(c->work));
        if (hctl[2] & 4) {
            c->dead = true;
            throw Err{FDTD_ERR_TIMEOUT, "a wait of the step kernel gave up after its time limit"};
        }
        if (hctl[2] & 1) {
            c->dead = true;
            throw Err{FDTD_ERR_UNSTABLE, "non-finite or exploding field during the run"};
        }
        if (hctl[0] != M) throw Err{FDTD_ERR_CUDA, "device step counter " + std::to_string(hctl[0]) + " != " + std::to_string(M)};
    }

    double forward(double* gap_out)
    {
        run(0);
        return forward_epilogue(gap_out);
    }

    // After a forward run: the gap DFT to the host and the objective F = sum_f w_f sum_gap |Ehat|^2.
    double forward_epilogue(double* gap_out)
    {
        const fdtd_grid_desc& d = c->d;
        const size_t ns = c->ngap * 3 * d.n_freq;
        gap_dft.assign(2 * ns, 0.0);
        double F = 0.0;
        if (ns) {
            CK(fdtd::launch_gap_gather(dft[0], (long long)c->nd, d.n_freq, base.db, base.dnx, base.dny, base.gb, gapbuf, c->work));
            c->tim.launches++;
            CK(cudaMemcpyAsync(gap_dft.data(), gapbuf, ns * sizeof(double2), cudaMemcpyDeviceToHost, c->work));
            CK(cudaStreamSynchronize(c->work));
            for (int f = 0; f < d.n_freq; ++f) {
                double s = 0.0;
                for (size_t q = 0; q < 3 * c->ngap; ++q) {
                    const double re = gap_dft[2 * (f * 3 * c->ngap + q)], im = gap_dft[2 * (f * 3 * c->ngap + q) + 1];
                    s += re * re + im * im;
                }
                F += c->weights[f] * s;
            }
        }
        if (gap_out && ns) std::memcpy(gap_out, gap_dft.data(), 2 * ns * sizeof(double));
        return F;
    }

    // Adjoint drive: 2F basis pulses b_q(t) = g(t) {cos, sin}(w_f (t - t0a)) and, per gap sample,
    // the real coefficients r_g with sum_q r_{g,q} Bhat_q(w_f) = w_f conj(Ehat_g(w_f)).
    void adjoint()
    {
        adjoint_drive();
        run(1);
    }

    // Build and upload the adjoint drive from the forward gap DFT (the part of the adjoint before its run).
    void adjoint_drive()
    {
        const fdtd_grid_desc& d = c->d;
        const int F = d.n_freq, nb = 2 * F, M = d.n_steps;
        if (!c->ngap) arg_error("the adjoint run needs a non-empty gap box");
        const double tau = d.adj_tau > 0.0 ? d.adj_tau : src_tau(d);
        const double t0 = 4.0 * tau;
        std::vector<double> wave((size_t)M * nb);
        for (int s = 0; s < M; ++s) {
            const double x = (s + 0.5) * c->dt - t0;
            const double env = std::exp(-x * x / (2.0 * tau * tau));
            for (int f = 0; f < F; ++f) {
                const double w = 2.0 * kPi * c->freqs[f];
                wave[(size_t)s * nb + 2 * f] = env * std::cos(w * x);
                wave[(size_t)s * nb + 2 * f + 1] = env * std::sin(w * x);
            }
        }
        // A[row][q]: rows (Re f, Im f) of sum_n b_q((n+1/2)dt) e^{-j w_f n dt}
        std::vector<double> A((size_t)nb * nb, 0.0);
        for (int f = 0; f < F; ++f) {
            const double w = 2.0 * kPi * c->freqs[f] * c->dt;
            for (int s = 0; s < M; ++s) {
                const double cr = std::cos(w * s), ci = -std::sin(w * s);
                for (int q = 0; q < nb; ++q) {
                    const double b = wave[(size_t)s * nb + q];
                    A[(2 * f) * nb + q] += b * cr;
                    A[(2 * f + 1) * nb + q] += b * ci;
                }
            }
        }
        double anorm = 0.0;                 // 1-norm, for the condition estimate below
        for (int q = 0; q < nb; ++q) {
            double col = 0.0;
            for (int r0 = 0; r0 < nb; ++r0) col += std::fabs(A[r0 * nb + q]);
            anorm = std::max(anorm, col);
        }
        // LU with partial pivoting, reused for every gap sample
        std::vector<int> piv(nb);
        for (int col = 0; col < nb; ++col) {
            int pr = col;
            for (int r = col + 1; r < nb; ++r)
                if (std::fabs(A[r * nb + col]) > std::fabs(A[pr * nb + col])) pr = r;
            if (A[pr * nb + col] == 0.0) arg_error("adjoint basis matrix is singular (try another adj_tau)");
            piv[col] = pr;
            if (pr != col)
                for (int q = 0; q < nb; ++q) std::swap(A[col * nb + q], A[pr * nb + q]);
            for (int r = col + 1; r < nb; ++r) {
                A[r * nb + col] /= A[col * nb + col];
                for (int q = col + 1; q < nb; ++q) A[r * nb + q] -= A[r * nb + col] * A[col * nb + q];
            }
        }
        auto lu_solve = [&](std::vector<double>& x) {
            for (int col = 0; col < nb; ++col) std::swap(x[col], x[piv[col]]);
            for (int row = 0; row < nb; ++row)
                for (int q = 0; q < row; ++q) x[row] -= A[row * nb + q] * x[q];
            for (int row = nb - 1; row >= 0; --row) {
                for (int q = row + 1; q < nb; ++q) x[row] -= A[row * nb + q] * x[q];
                x[row] /= A[row * nb + row];
            }
        };
        // cond_1 = |A|_1 |A^{-1}|_1; an ill-conditioned basis loses the adjoint drive's accuracy
        {
            double inorm = 0.0;
            std::vector<double> e(nb);
            std::vector<double> colsum(nb, 0.0);
            for (int q = 0; q < nb; ++q) {
                std::fill(e.begin(), e.end(), 0.0);
                e[q] = 1.0;
                lu_solve(e);
                double cs = 0.0;
                for (int r0 = 0; r0 < nb; ++r0) cs += std::fabs(e[r0]);
                inorm = std::max(inorm, cs);
            }
            adj_cond = anorm * inorm;
            const double limit = sizeof(T) == 4 ? 1e4 : 1e10;
            if (!(adj_cond <= limit))
                arg_error("adjoint basis too ill-conditioned for this precision (cond " + std::to_string(adj_cond) +
                          "): lengthen n_steps, raise adj_tau, or spread the objective frequencies");
        }
        const size_t ns = c->ngap * 3;
        std::vector<T> r(ns * nb);
        std::vector<double> rhs(nb);
        for (int cc = 0; cc < 3; ++cc)
            for (size_t gv = 0; gv < c->ngap; ++gv) {
                for (int f = 0; f < F; ++f) {
                    const size_t o = 2 * ((size_t)(f * 3 + cc) * c->ngap + gv);
                    rhs[2 * f] = c->weights[f] * gap_dft[o];
                    rhs[2 * f + 1] = -c->weights[f] * gap_dft[o + 1];
                }
                lu_solve(rhs);
                for (int q = 0; q < nb; ++q) r[(gv * 3 + cc) * nb + q] = (T)rhs[q];
            }
        std::vector<T> wt(wave.size());
        for (size_t q = 0; q < wave.size(); ++q) wt[q] = (T)wave[q];
        CK(cudaMemcpyAsync(src_wave[1], wt.data(), wt.size() * sizeof(T), cudaMemcpyHostToDevice, c->work));
        CK(cudaMemcpyAsync(src_r[1], r.data(), r.size() * sizeof(T), cudaMemcpyHostToDevice, c->work));
        CK(cudaStreamSynchronize(c->work));
        if (pa.nb != nb || pa.src_r != src_r[1]) {
            pa.nb = nb;
            pa.src_r = src_r[1];
            pa.src_wave = src_wave[1];
            std::memcpy(pa.sb, base.gb, sizeof pa.sb);
            refresh_params();
        }
    }

    // ---- batched runs (fdtd_batch_*) --------------------------------------------------------------
    // Start a run of the given mode inside a batch: zero the state (on the handle's stream) and describe
    // the run for the persistent kernel; the adjoint mode first builds its drive, as fdtd_adjoint does.
    void batch_prepare(int mode, fdtd::BatchSlot<T>* slot)
    {
        if (mode == 1) adjoint_drive();
        reset_state(mode);
        const KParams<T>& p = mode ? pa : pf;
        slot->kp[0] = par(p, 0);
        slot->kp[1] = par(p, 1);
        slot->dp = dp[mode];
        batch_shape(c->d, &slot->sz, &slot->cw);
        slot->nslab = (c->d.nz + slot->sz - 1) / slot->sz;
        slot->nxyc = (int)(((long long)c->d.nx * c->d.ny + slot->cw - 1) / slot->cw);
        slot->n0 = 0;
    }

    // Flags of a finished batched run (the device flags the kernels raise): throws like run().
    void batch_check()
    {
        int hctl[4];
        CK(cudaMemcpyAsync(hctl, ctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->work));
        CK(cudaStreamSynchronize(c->work));
        if (hctl[2] & 1) {
            c->dead = true;
            throw Err{FDTD_ERR_UNSTABLE, "non-finite or exploding field during the run"};
        }
    }

    void gradient(void* out, int dtype, int on_device)
    {
        const size_t nd = c->nd;
        GParams<T> g{};
        std::memcpy(g.db, base.db, sizeof g.db);
        std::memcpy(g.gb, base.gb, sizeof g.gb);
        g.dnx = base.dnx;
        g.dny = base.dny;
        g.nd = (long long)nd;
        g.nf = c->d.n_freq;
        g.dft_f = dft[0];
        g.dft_a = dft[1];
        g.AB = AB;
        g.rho = rho;
        g.per_comp = c->d.density_layout == 1 ? 1 : 0;
        g.nout = (long long)c->nvar;
        std::memcpy(g.off, c->voff, sizeof g.off);
        std::memcpy(g.mdim, c->vdim, sizeof g.mdim);
        for (int cc = 0; cc < 3; ++cc) g.rhoc[cc] = base.rhoc[cc];
        g.grad64 = grad;
        g.grad32 = nullptr;
        float* grad32_dev = (float*)staging;
        if (on_device && out) {
            if (dtype == 1) g.grad64 = (double*)out;
            else g.grad32 = (float*)out;
        } else if (out && dtype == 0) {
            g.grad32 = grad32_dev;
        }
        g.partial = partial;
        g.counter = counter;
        const size_t nout = c->nvar;
        const unsigned nblk = (unsigned)((nout + fdtd::kReduceThreads - 1) / fdtd::kReduceThreads);
        if (nblk == 0) return;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (c->prof) {
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            CK(cudaEventRecord(e0, c->work));
        }
        CK(fdtd::launch_grad<T>(g, nblk, c->work));
        c->tim.launches++;
        c->tim.grad_launches++;
        if (c->prof) {
            CK(cudaEventRecord(e1, c->work));
            CK(cudaEventSynchronize(e1));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            c->tim.grad_ms += ms;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
        if (out && !on_device) {   // straight into the caller's (pageable or pinned) buffer
            if (dtype == 1)
                CK(cudaMemcpyAsync(out, grad, nout * sizeof(double), cudaMemcpyDeviceToHost, c->work));
            else
                CK(cudaMemcpyAsync(out, grad32_dev, nout * sizeof(float), cudaMemcpyDeviceToHost, c->work));
            CK(cudaStreamSynchronize(c->work));
        }
    }

    double grad_norm2()
    {
        const unsigned nblk = (unsigned)((c->nvar + fdtd::kReduceThreads - 1) / fdtd::kReduceThreads);
        double v = 0.0;
        CK(cudaMemcpyAsync(&v, partial + nblk, sizeof(double), cudaMemcpyDeviceToHost, c->work));
        CK(cudaStreamSynchronize(c->work));
        return v;
    }

    // Field / DFT copies: to a host buffer (synchronous) or, on_device, to a device buffer on the
    // handle's stream (ordered after the last run, no host wait).
    void get_field(int which, double* dst, int on_device)
    {
        T* src = cur_field(which);
        if (on_device) {
            CK(fdtd::launch_to_double<T>(src, (long long)c->ncell, dst, c->work));
            c->tim.launches++;
            return;
        }
        std::vector<T> h(c->ncell);
        CK(cudaMemcpyAsync(h.data(), src, c->ncell * sizeof(T), cudaMemcpyDeviceToHost, c->work));
        CK(cudaStreamSynchronize(c->work));
        for (size_t q = 0; q < c->ncell; ++q) dst[q] = (double)h[q];
    }

    void get_dft(int adjoint, double* dst, int on_device)
    {
        CK(cudaMemcpyAsync(dst, dft[adjoint ? 1 : 0], c->nd * 3 * c->d.n_freq * sizeof(double2),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->work));
        if (!on_device) CK(cudaStreamSynchronize(c->work));
    }

    // Failure-path test hook: with timeout_ns > 0, block (0, 0, 0) of the interior kernel at step 0
    // of every later run waits, with that limit, on an mbarrier that no copy completes (0: off).
    void set_stall(long long timeout_ns)
    {
        base.stall_ns = timeout_ns;
        refresh_params();
    }

    // dY/drho constants of the last set_materials: [3][n_freq] x (A.re, A.im, B.re, B.im).
    void gradient_constants(double* dst) const
    {
        for (size_t q = 0; q < ab_host.size(); ++q) {
            dst[2 * q] = ab_host[q].x;
            dst[2 * q + 1] = ab_host[q].y;
        }
    }

    void index_map(int which, int32_t* dst, size_t n)
    {
        int32_t* dev = nullptr;
        CK(cudaMallocFromPoolAsync((void**)&dev, n * sizeof(int32_t), device_pool(c->device), c->work));
        cudaError_t e = fdtd::launch_index_map<T>(pf, which, dev, c->work);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, dev, n * sizeof(int32_t), cudaMemcpyDeviceToHost, c->work);
        cudaFreeAsync(dev, c->work);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->work);
        c->tim.launches++;
        CK(e);
    }
};

// ---------------------------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------------------------
namespace {

thread_local std::string g_last_error;   // errors of calls without a (live) handle

template <typename F>
fdtd_status guarded(fdtd_ctx* c, F&& fn)
{
    try {
        fn();
        return FDTD_OK;
    } catch (const Err& e) {
        g_last_error = e.msg;
        if (c) {
            c->err = e.msg;
            if (e.code == FDTD_ERR_CUDA) c->dead = true;
        }
        return e.code;
    } catch (const std::bad_alloc&) {
        if (c) c->err = "host allocation failed";
        return FDTD_ERR_OOM;
    } catch (...) {
        if (c) c->err = "unexpected exception";
        return FDTD_ERR_CUDA;
    }
}

template <typename T>
Solver<T>* as(fdtd_ctx* c) { return static_cast<Solver<T>*>(c->impl.get()); }

}  // namespace

namespace fdtd {
// Error text for handle-less calls in other translation units (read by fdtd_last_error(NULL)).
void set_thread_error(const std::string& msg) { g_last_error = msg; }
}  // namespace fdtd

namespace {

// Dispatch on the handle's precision.
template <typename F>
void dispatch(fdtd_ctx* c, F&& fn)
{
    if (c->d.precision == 64)
        fn(as<double>(c));
    else
        fn(as<float>(c));
}

void enter(fdtd_ctx* c)
{
    CK(cudaSetDevice(c->device));
    CK(cudaEventRecord(c->fence, c->user));
    CK(cudaStreamWaitEvent(c->work, c->fence, 0));
}

void leave(fdtd_ctx* c)
{
    CK(cudaEventRecord(c->fence, c->work));
    CK(cudaStreamWaitEvent(c->user, c->fence, 0));
}

fdtd_status check_handle(fdtd_handle h, bool allow_dead = false)
{
    if (!h) return FDTD_ERR_ARG;
    if (h->dead && !allow_dead) return FDTD_ERR_STATE;
    if (h->batch && !allow_dead) {   // a run of this handle is in a batch: only inspection until it ends
        h->err = "a run of this handle is in progress in a batch";
        return FDTD_ERR_STATE;
    }
    return FDTD_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Batches: several runs advanced together by one persistent kernel (fdtd_batch.cu)
// ---------------------------------------------------------------------------------------------
struct fdtd_batch_ctx {
    int device = 0;
    cudaStream_t user = nullptr, stream = nullptr;
    cudaEvent_t fence = nullptr;
    fdtd::BatchSlot<float>* slots = nullptr;    // [kMaxBatch] on the device
    unsigned* prog = nullptr;                   // [kMaxBatch][kMaxBatchSlabs]
    unsigned long long* ticket = nullptr;
    int* err = nullptr;                         // [2]
    int* gate = nullptr;                        // test hook flag, stays 0
    bool use_gate = false;
    unsigned long long wait_ns = 1000000000ull; // one second
    struct Run {
        fdtd_ctx* h = nullptr;
        int mode = 0, done = 0, M = 0;
    };
    Run runs[fdtd::kMaxBatch];
    cudaGraph_t graph[3] = {nullptr, nullptr, nullptr};       // per pole bucket 4 / 8 / 16 (kept: the
    cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};   // kernel node is updated through it)
    cudaGraphNode_t knode[3] = {nullptr, nullptr, nullptr};
    unsigned blocks[3] = {0, 0, 0};
    long long launches = 0;
    bool dead = false;
    std::string err_msg;
    std::vector<void*> allocs;
    std::mutex mu;                               // fdtd_destroy of a member handle may come from any thread
};

namespace {

int bucket_index(int bucket) { return bucket <= 4 ? 0 : (bucket <= 8 ? 1 : 2); }

void batch_detach(fdtd_ctx* h)
{
    fdtd_batch_ctx* b = h->batch;
    if (!b) return;
    std::lock_guard<std::mutex> lock(b->mu);
    cudaStreamSynchronize(b->stream);           // no launch of the batch may still touch the handle
    if (h->batch_slot >= 0) b->runs[h->batch_slot] = fdtd_batch_ctx::Run{};
    h->batch = nullptr;
    h->batch_slot = -1;
}

// The launch's graph for one pole bucket: zero the ticket counter and the error words, then the kernel.
// Captured once; every launch only rewrites the kernel's parameter block.
void batch_graph(fdtd_batch_ctx* b, int bi, const fdtd::BatchLaunch& L)
{
    const void* fn = fdtd::batch_kernel_fn<float>(bi == 0 ? 4 : (bi == 1 ? 8 : 16));
    cudaKernelNodeParams kp{};
    kp.func = (void*)fn;
    kp.gridDim = dim3(b->blocks[bi]);
    kp.blockDim = dim3(fdtd::kBatchThreads);
    kp.sharedMemBytes = 0;
    void* args[1] = {(void*)&L};
    kp.kernelParams = args;
    if (!b->exec[bi]) {
        cudaGraph_t g = nullptr;
        CK(cudaGraphCreate(&g, 0));
        cudaGraphNode_t m1 = nullptr, m2 = nullptr, k = nullptr;
        cudaMemsetParams ms{};
        ms.dst = b->ticket;
        ms.value = 0;
        ms.elementSize = 4;
        ms.width = 2;                         // one unsigned long long
        ms.height = 1;
        cudaError_t e = cudaGraphAddMemsetNode(&m1, g, nullptr, 0, &ms);
        ms.dst = b->err;
        if (e == cudaSuccess) e = cudaGraphAddMemsetNode(&m2, g, &m1, 1, &ms);
        if (e == cudaSuccess) e = cudaGraphAddKernelNode(&k, g, &m2, 1, &kp);
        cudaGraphExec_t ex = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            CK(e);
        }
        b->graph[bi] = g;
        b->exec[bi] = ex;
        b->knode[bi] = k;
    } else {
        CK(cudaGraphExecKernelNodeSetParams(b->exec[bi], b->knode[bi], &kp));
    }
}

}  // namespace

extern "C" {

fdtd_status fdtd_batch_create(void* cuda_stream, fdtd_batch* out)
{
    if (!out) return FDTD_ERR_ARG;
    *out = nullptr;
    fdtd_batch_ctx* b = new (std::nothrow) fdtd_batch_ctx();
    if (!b) return FDTD_ERR_OOM;
    fdtd_status st = guarded(nullptr, [&] {
        CK(cudaGetDevice(&b->device));
        b->user = (cudaStream_t)cuda_stream;
        CK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&b->fence, cudaEventDisableTiming));
        auto alloc = [&](size_t n) {
            void* p = nullptr;
            if (cudaMallocFromPoolAsync(&p, n, device_pool(b->device), b->stream) != cudaSuccess) {
                cudaGetLastError();
                throw Err{FDTD_ERR_OOM, "batch: device allocation failed"};
            }
            b->allocs.push_back(p);
            return p;
        };
        b->slots = (fdtd::BatchSlot<float>*)alloc(sizeof(fdtd::BatchSlot<float>) * fdtd::kMaxBatch);
        b->prog = (unsigned*)alloc(sizeof(unsigned) * fdtd::kMaxBatch * fdtd::kMaxBatchSlabs);
        b->ticket = (unsigned long long*)alloc(256);
        b->err = (int*)alloc(256);
        b->gate = (int*)alloc(256);
        CK(cudaMemsetAsync(b->err, 0, 256, b->stream));
        CK(cudaMemsetAsync(b->gate, 0, 256, b->stream));
        int sms = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
        for (int bi = 0; bi < 3; ++bi) {
            int per = 0;
            CK(fdtd::batch_blocks_per_sm<float>(bi == 0 ? 4 : (bi == 1 ? 8 : 16), &per));
            b->blocks[bi] = (unsigned)std::max(1, sms * std::max(1, per));
        }
        CK(cudaStreamSynchronize(b->stream));
    });
    if (st != FDTD_OK) {
        fdtd_batch_destroy(b);
        return st;
    }
    *out = b;
    return FDTD_OK;
}

fdtd_status fdtd_batch_submit(fdtd_batch b, fdtd_handle h, int adjoint)
{
    if (!b || (adjoint != 0 && adjoint != 1)) return FDTD_ERR_ARG;
    if (b->dead) {
        g_last_error = "batch is dead after a failed launch";
        return FDTD_ERR_STATE;
    }
    if (fdtd_status s = check_handle(h)) return s;
    if (h->device != b->device || h->d.precision != 32) {
        h->err = "batch: the handle must be an FP32 handle on the batch's device";
        return FDTD_ERR_ARG;
    }
    if (adjoint ? !h->has_fwd : (!h->has_mat || (h->nd && !h->has_rho))) {
        h->err = adjoint ? "batched adjoint before forward" : "set_materials and set_density first";
        return FDTD_ERR_STATE;
    }
    int bsz = 0, bcw = 0;
    batch_shape(h->d, &bsz, &bcw);
    const long long nslab = (h->d.nz + bsz - 1) / bsz;
    const long long nxyc = ((long long)h->d.nx * h->d.ny + bcw - 1) / bcw;
    if (2LL * h->d.n_steps * nxyc >= (1LL << 32) || nslab > fdtd::kMaxBatchSlabs) {
        h->err = "batch: grid or step count too large for the batch's work-item counters";
        return FDTD_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(b->mu);
    int slot = -1;
    for (int q = 0; q < fdtd::kMaxBatch; ++q)
        if (!b->runs[q].h) {
            slot = q;
            break;
        }
    if (slot < 0) {
        h->err = "batch: all " + std::to_string(fdtd::kMaxBatch) + " slots are in use";
        return FDTD_ERR_STATE;
    }
    h->cancel.store(0);
    return guarded(h, [&] {
        enter(h);
        fdtd::BatchSlot<float> hs{};
        as<float>(h)->batch_prepare(adjoint, &hs);
        hs.prog = b->prog + (size_t)slot * fdtd::kMaxBatchSlabs;
        CK(cudaMemsetAsync(hs.prog, 0, sizeof(unsigned) * hs.nslab, h->work));
        CK(cudaMemcpyAsync(b->slots + slot, &hs, sizeof hs, cudaMemcpyHostToDevice, h->work));
        CK(cudaEventRecord(h->bfence, h->work));
        CK(cudaStreamWaitEvent(b->stream, h->bfence, 0));
        CK(cudaStreamSynchronize(h->work));     // the slot description above lives on this stack
        if (adjoint)
            h->has_adj = h->has_grad = false;
        else
            h->has_fwd = h->has_adj = h->has_grad = false;
        b->runs[slot] = fdtd_batch_ctx::Run{h, adjoint, 0, h->d.n_steps};
        h->batch = b;
        h->batch_slot = slot;
    });
}

fdtd_status fdtd_batch_run(fdtd_batch b, int max_steps, fdtd_handle* done, fdtd_status* done_status, int capacity,
                           int* n_done)
{
    if (!b || max_steps < 1 || !n_done || capacity < 0 || (capacity > 0 && (!done || !done_status))) return FDTD_ERR_ARG;
    *n_done = 0;
    if (b->dead) {
        g_last_error = "batch is dead after a failed launch";
        return FDTD_ERR_STATE;
    }
    std::lock_guard<std::mutex> lock(b->mu);
    struct Act {
        int slot, nph, cnt;
        long long items;
        int bucket;
    };
    std::vector<Act> act;
    for (int q = 0; q < fdtd::kMaxBatch; ++q) {
        const auto& r = b->runs[q];
        if (!r.h) continue;
        const int cnt = std::min(max_steps, r.M - r.done);
        int bsz = 0, bcw = 0;
        batch_shape(r.h->d, &bsz, &bcw);
        const long long nslab = (r.h->d.nz + bsz - 1) / bsz;
        const long long nxyc = ((long long)r.h->d.nx * r.h->d.ny + bcw - 1) / bcw;
        act.push_back(Act{q, 2 * cnt, cnt, nslab * nxyc, as<float>(r.h)->bucket});
    }
    if (act.empty()) return FDTD_OK;
    if ((int)act.size() > capacity) {   // every run may finish in this launch
        g_last_error = "batch: capacity below the number of runs in the batch";
        return FDTD_ERR_ARG;
    }
    std::stable_sort(act.begin(), act.end(), [](const Act& a, const Act& c) { return a.nph > c.nph; });
    fdtd::BatchLaunch L{};
    L.nruns = (int)act.size();
    L.pre[0] = 0;
    int bucket = 4;
    for (int j = 0; j < L.nruns; ++j) {
        L.slot[j] = act[j].slot;
        L.pre[j + 1] = L.pre[j] + act[j].items;
        bucket = std::max(bucket, act[j].bucket);
    }
    // segments of rounds with the same number of taking-part runs (a prefix of the sorted list)
    int g = 0, nseg = 0;
    long long t0 = 0;
    for (int m = L.nruns; m > 0; --m) {
        const int g1 = act[m - 1].nph;       // runs 0 .. m-1 take part in rounds [g, g1)
        if (g1 <= g) continue;
        L.seg_g0[nseg] = g;
        L.seg_m[nseg] = m;
        L.seg_t0[nseg] = t0;
        t0 += (long long)(g1 - g) * L.pre[m];
        g = g1;
        ++nseg;
    }
    L.nseg = nseg;
    L.seg_g0[nseg] = g;
    L.seg_t0[nseg] = t0;
    L.slots = b->slots;
    L.ticket = b->ticket;
    L.err = b->err;
    L.gate = b->use_gate ? b->gate : nullptr;
    L.wait_ns = b->wait_ns;
    return guarded(nullptr, [&] {
        CK(cudaSetDevice(b->device));
        CK(cudaEventRecord(b->fence, b->user));
        CK(cudaStreamWaitEvent(b->stream, b->fence, 0));
        std::vector<int> n0(act.size());
        for (size_t j = 0; j < act.size(); ++j) {
            n0[j] = b->runs[act[j].slot].done;
            CK(cudaMemcpyAsync(&b->slots[act[j].slot].n0, &n0[j], sizeof(int), cudaMemcpyHostToDevice, b->stream));
        }
        const int bi = bucket_index(bucket);
        batch_graph(b, bi, L);
        CK(cudaGraphLaunch(b->exec[bi], b->stream));
        b->launches++;
        int herr[2] = {0, 0};
        CK(cudaMemcpyAsync(herr, b->err, sizeof herr, cudaMemcpyDeviceToHost, b->stream));
        CK(cudaStreamSynchronize(b->stream));
        if (herr[0]) {
            b->dead = true;
            for (auto& r : b->runs)
                if (r.h) {
                    r.h->dead = true;
                    r.h->err = "batch: a dependency wait of the persistent kernel gave up after its time limit";
                    r.h->batch = nullptr;
                    r.h->batch_slot = -1;
                    r = fdtd_batch_ctx::Run{};
                }
            throw Err{FDTD_ERR_TIMEOUT, "batch: a dependency wait of the persistent kernel gave up after its time limit "
                                        "(work item " + std::to_string(herr[1]) + ")"};
        }
        for (const Act& a : act) {
            auto& r = b->runs[a.slot];
            r.done += a.cnt;
            if (r.done < r.M) continue;
            fdtd_ctx* h = r.h;
            const int mode = r.mode;
            r = fdtd_batch_ctx::Run{};
            h->batch = nullptr;
            h->batch_slot = -1;
            h->tim.launches += 1;
            const fdtd_status st = guarded(h, [&] {
                CK(cudaEventRecord(b->fence, b->stream));
                CK(cudaStreamWaitEvent(h->work, b->fence, 0));
                Solver<float>* s = as<float>(h);
                s->batch_check();
                if (mode == 0) {
                    h->F_last = s->forward_epilogue(nullptr);
                    h->has_fwd = true;
                } else {
                    h->has_adj = true;
                }
                leave(h);
            });
            done[*n_done] = h;
            done_status[*n_done] = st;
            ++*n_done;
        }
        CK(cudaEventRecord(b->fence, b->stream));
        CK(cudaStreamWaitEvent(b->user, b->fence, 0));
    });
}

fdtd_status fdtd_batch_set_wait_limit(fdtd_batch b, long long wait_ns, int gate)
{
    if (!b || wait_ns <= 0 || wait_ns > 60LL * 1000 * 1000 * 1000 || (gate != 0 && gate != 1)) return FDTD_ERR_ARG;
    std::lock_guard<std::mutex> lock(b->mu);
    b->wait_ns = (unsigned long long)wait_ns;
    b->use_gate = gate != 0;
    return FDTD_OK;
}

fdtd_status fdtd_batch_set_blocks(fdtd_batch b, int blocks)
{
    if (!b || blocks < 0) return FDTD_ERR_ARG;
    std::lock_guard<std::mutex> lock(b->mu);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) return FDTD_ERR_CUDA;
    for (int bi = 0; bi < 3; ++bi) {
        int per = 0;
        if (fdtd::batch_blocks_per_sm<float>(bi == 0 ? 4 : (bi == 1 ? 8 : 16), &per) != cudaSuccess) return FDTD_ERR_CUDA;
        const unsigned full = (unsigned)std::max(1, sms * std::max(1, per));
        b->blocks[bi] = blocks == 0 ? full : std::min(full, (unsigned)blocks);
        if (b->exec[bi]) {                       // the grid size is part of the captured graph
            cudaGraphExecDestroy(b->exec[bi]);
            cudaGraphDestroy(b->graph[bi]);
            b->exec[bi] = nullptr;
            b->graph[bi] = nullptr;
            b->knode[bi] = nullptr;
        }
    }
    return FDTD_OK;
}

fdtd_status fdtd_batch_info(fdtd_batch b, int* n_runs, long long* launches)
{
    if (!b) return FDTD_ERR_ARG;
    std::lock_guard<std::mutex> lock(b->mu);
    int n = 0;
    for (const auto& r : b->runs) n += r.h ? 1 : 0;
    if (n_runs) *n_runs = n;
    if (launches) *launches = b->launches;
    return FDTD_OK;
}

fdtd_status fdtd_batch_destroy(fdtd_batch b)
{
    if (!b) return FDTD_ERR_ARG;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    {
        std::lock_guard<std::mutex> lock(b->mu);
        for (auto& r : b->runs)
            if (r.h) {
                r.h->batch = nullptr;
                r.h->batch_slot = -1;
                r = fdtd_batch_ctx::Run{};
            }
    }
    for (auto& e : b->exec)
        if (e) cudaGraphExecDestroy(e);
    for (auto& g : b->graph)
        if (g) cudaGraphDestroy(g);
    if (b->stream) {
        for (void* p : b->allocs) cudaFreeAsync(p, b->stream);
        cudaStreamSynchronize(b->stream);
        cudaStreamDestroy(b->stream);
    }
    if (b->fence) cudaEventDestroy(b->fence);
    delete b;
    return FDTD_OK;
}

fdtd_status fdtd_get_objective(fdtd_handle h, double* F_out, double* gap_dft_out)
{
    if (fdtd_status s = check_handle(h, true)) return s;
    if (!h->has_fwd) {
        h->err = "no forward result";
        return FDTD_ERR_STATE;
    }
    return guarded(h, [&] {
        if (F_out) *F_out = h->F_last;
        if (gap_dft_out)
            dispatch(h, [&](auto* s) { std::memcpy(gap_dft_out, s->gap_dft.data(), s->gap_dft.size() * sizeof(double)); });
    });
}

fdtd_status fdtd_footprint_bytes(const fdtd_grid_desc* desc, const int p_total[3], size_t* bytes)
{
    if (!desc || !p_total || !bytes) return FDTD_ERR_ARG;
    return guarded(nullptr, [&] {
        validate(*desc);
        *bytes = footprint(*desc, p_total);
    });
}

fdtd_status fdtd_create_grid(const fdtd_grid_desc* desc, void* cuda_stream, fdtd_handle* out)
{
    if (!desc || !out) return FDTD_ERR_ARG;
    *out = nullptr;
    fdtd_ctx* c = new (std::nothrow) fdtd_ctx();
    if (!c) return FDTD_ERR_OOM;
    fdtd_status st = guarded(c, [&] {
        validate(*desc);
        c->d = *desc;
        std::memcpy(c->dbu, desc->design_box, sizeof c->dbu);
        c->nvar = design_vars(*desc, c->voff, c->vdim);
        working_box(*desc, c->d.design_box);
        c->freqs.assign(desc->freqs_hz, desc->freqs_hz + desc->n_freq);
        c->weights.assign(desc->n_freq, 1.0);
        if (desc->freq_weights) c->weights.assign(desc->freq_weights, desc->freq_weights + desc->n_freq);
        c->d.freqs_hz = c->freqs.data();
        c->d.freq_weights = c->weights.data();
        if (desc->src_wave) {
            c->wave.assign(desc->src_wave, desc->src_wave + 2 * (size_t)desc->n_steps + 1);
            c->d.src_wave = c->wave.data();
        }
        CK(cudaGetDevice(&c->device));
        c->user = (cudaStream_t)cuda_stream;
        CK(cudaStreamCreateWithFlags(&c->work, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->fence, cudaEventDisableTiming));
        CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->bfence, cudaEventDisableTiming));
        c->dt = desc->courant * desc->dx / kC0;
        c->ncell = (size_t)desc->nx * desc->ny * desc->nz;
        c->nd = (size_t)box_count(c->d.design_box);
        c->ngap = (size_t)box_count(desc->gap_box);
        for (int a = 0; a < 3; ++a) {
            c->dn[a] = c->nd ? c->d.design_box[2 * a + 1] - c->d.design_box[2 * a] : 0;
            c->gn[a] = c->ngap ? desc->gap_box[2 * a + 1] - desc->gap_box[2 * a] : 0;
        }
    });
    if (st != FDTD_OK) {
        fdtd_destroy(c);
        return st;
    }
    *out = c;
    return FDTD_OK;
}

fdtd_status fdtd_set_materials(fdtd_handle h, const fdtd_ccpr_material* bg, const fdtd_ccpr_material* m1,
                               const fdtd_ccpr_material* m2, double gamma)
{
    if (fdtd_status s = check_handle(h)) return s;
    return guarded(h, [&] {
        const Material B = import_material(bg, "bg"), A1 = import_material(m1, "m1"), A2 = import_material(m2, "m2");
        for (int k = 0; k < 3; ++k)
            if (!B.poles[k].empty()) arg_error("background material must be non-dispersive (no poles)");
        int pt[3];
        for (int k = 0; k < 3; ++k) {
            pt[k] = (int)(A1.poles[k].size() + A2.poles[k].size());
            if (pt[k] > fdtd::kMaxPoles) arg_error("more than 16 poles on one component (m1 + m2)");
        }
        CK(cudaSetDevice(h->device));
        if (!h->impl) {
            if (h->d.precision == 64) {
                auto* s = new Solver<double>(h);
                h->impl.reset(s);
                s->allocate(pt);
            } else {
                auto* s = new Solver<float>(h);
                h->impl.reset(s);
                s->allocate(pt);
            }
        }
        dispatch(h, [&](auto* s) { s->set_materials(B, A1, A2, gamma); });
        CK(cudaStreamSynchronize(h->work));
        h->has_mat = true;
        h->has_fwd = h->has_adj = h->has_grad = false;
    });
}

fdtd_status fdtd_set_density(fdtd_handle h, const void* rho, size_t n, int dtype, int on_device)
{
    if (fdtd_status s = check_handle(h)) return s;
    if (!h->has_mat) {
        h->err = "set_materials first";
        return FDTD_ERR_STATE;
    }
    if (n != h->nvar || (dtype != 0 && dtype != 1) || (!rho && n)) {
        h->err = "density size/dtype mismatch: expected " + std::to_string(h->nvar) + " values";
        return FDTD_ERR_ARG;
    }
    return guarded(h, [&] {
        enter(h);
        if (n) dispatch(h, [&](auto* s) { s->set_density(rho, dtype, on_device); });
        leave(h);
        h->has_rho = true;
        h->has_fwd = h->has_adj = h->has_grad = false;
    });
}

fdtd_status fdtd_forward(fdtd_handle h, double* F_out, double* gap_dft_out)
{
    if (fdtd_status s = check_handle(h)) return s;
    if (!h->has_mat || (h->nd && !h->has_rho)) {
        h->err = "set_materials and set_density first";
        return FDTD_ERR_STATE;
    }
    h->cancel.store(0);
    return guarded(h, [&] {
        enter(h);
        double F = 0.0;
        dispatch(h, [&](auto* s) { F = s->forward(gap_dft_out); });
        leave(h);
        if (F_out) *F_out = F;
        h->F_last = F;
        h->has_fwd = true;
        h->has_adj = h->has_grad = false;
    });
}

fdtd_status fdtd_adjoint(fdtd_handle h)
{
    if (fdtd_status s = check_handle(h)) return s;
    if (!h->has_fwd) {
        h->err = "adjoint before forward";
        return FDTD_ERR_STATE;
    }
    h->cancel.store(0);
    return guarded(h, [&] {
        enter(h);
        dispatch(h, [&](auto* s) { s->adjoint(); });
        leave(h);
        h->has_adj = true;
    });
}

fdtd_status fdtd_gradient(fdtd_handle h, void* grad, size_t n, int dtype, int on_device)
{
    if (fdtd_status s = check_handle(h)) return s;
    if (!h->has_adj) {
        h->err = "gradient before adjoint";
        return FDTD_ERR_STATE;
    }
    if ((grad && n != h->nvar) || (dtype != 0 && dtype != 1)) {
        h->err = "gradient buffer size/dtype mismatch";
        return FDTD_ERR_ARG;
    }
    return guarded(h, [&] {
        enter(h);
        dispatch(h, [&](auto* s) { s->gradient(grad, dtype, on_device); });
        leave(h);
        h->has_grad = true;
    });
}

fdtd_status fdtd_paper_forward(fdtd_handle h, int checkpoint_steps, double* F_out)
{
    if (fdtd_status s = check_handle(h)) return s;
    if (!h->has_rho) {
        h->err = "paper forward before density";
        return FDTD_ERR_STATE;
    }
    return guarded(h, [&] {
        enter(h);
        double F = 0.0;
        dispatch(h, [&](auto* s) { F = s->paper_forward(checkpoint_steps); });
        leave(h);
        if (F_out) *F_out = F;
    });
}

fdtd_status fdtd_paper_gradient(fdtd_handle h, int pole_pairing, void* grad, size_t n, int dtype, int on_device)
{
    if (fdtd_status s = check_handle(h)) return s;
    if ((grad && n != h->nd) || (dtype != 0 && dtype != 1) || (pole_pairing != 0 && pole_pairing != 1)) {
        h->err = "paper gradient: buffer size/dtype or pole_pairing mismatch";
        return FDTD_ERR_ARG;
    }
    return guarded(h, [&] {
        enter(h);
        dispatch(h, [&](auto* s) { s->paper_gradient(pole_pairing, grad, dtype, on_device); });
        leave(h);
    });
}

fdtd_status fdtd_gradient_norm(fdtd_handle h, double* out)
{
    if (fdtd_status s = check_handle(h)) return s;
    if (!h->has_grad || !out) return FDTD_ERR_STATE;
    return guarded(h, [&] { dispatch(h, [&](auto* s) { *out = s->grad_norm2(); }); });
}

fdtd_status fdtd_get_field(fdtd_handle h, int which, double* dst, size_t n, int on_device)
{
    if (fdtd_status s = check_handle(h, true)) return s;
    if (!h->impl || which < 0 || which > 5 || n != h->ncell || !dst) return FDTD_ERR_ARG;
    return guarded(h, [&] {
        if (on_device) enter(h);
        dispatch(h, [&](auto* s) { s->get_field(which, dst, on_device); });
        if (on_device) leave(h);
    });
}

fdtd_status fdtd_get_dft(fdtd_handle h, int adjoint, double* dst, size_t n_doubles, int on_device)
{
    if (fdtd_status s = check_handle(h, true)) return s;
    if (!h->impl || !dst || n_doubles != 2 * h->nd * 3 * (size_t)h->d.n_freq) return FDTD_ERR_ARG;
    return guarded(h, [&] {
        if (on_device) enter(h);
        dispatch(h, [&](auto* s) { s->get_dft(adjoint, dst, on_device); });
        if (on_device) leave(h);
    });
}

fdtd_status fdtd_get_gradient_constants(fdtd_handle h, double* dst, size_t n_doubles)
{
    if (fdtd_status s = check_handle(h, true)) return s;
    if (!h->impl || !h->has_mat) {
        h->err = "set_materials first";
        return FDTD_ERR_STATE;
    }
    if (!dst || n_doubles != 3 * 4 * (size_t)h->d.n_freq) {
        h->err = "gradient constants: expected 12 * n_freq doubles";
        return FDTD_ERR_ARG;
    }
    return guarded(h, [&] { dispatch(h, [&](auto* s) { s->gradient_constants(dst); }); });
}

fdtd_status fdtd_inject_wait_timeout(fdtd_handle h, long long timeout_ns)
{
    if (fdtd_status s = check_handle(h)) return s;
    if (!h->impl || !h->impl->has_interior()) {
        h->err = "the wait-timeout hook needs a grid with an interior box (fused step kernel)";
        return FDTD_ERR_ARG;
    }
    if (timeout_ns < 0 || timeout_ns > 10LL * 1000 * 1000 * 1000) {
        h->err = "timeout_ns must lie in [0, 1e10]";
        return FDTD_ERR_ARG;
    }
    return guarded(h, [&] { dispatch(h, [&](auto* s) { s->set_stall(timeout_ns); }); });
}

fdtd_status fdtd_get_index_map(fdtd_handle h, int which, int32_t* dst, size_t n)
{
    if (fdtd_status s = check_handle(h, true)) return s;
    if (!h->impl || !dst || which < 0 || which > 3) return FDTD_ERR_ARG;
    if (n != (which <= 1 ? 3 * h->ncell : h->ncell)) return FDTD_ERR_ARG;
    return guarded(h, [&] { dispatch(h, [&](auto* s) { s->index_map(which, dst, n); }); });
}

fdtd_status fdtd_set_profiling(fdtd_handle h, int on)
{
    if (fdtd_status s = check_handle(h)) return s;
    h->prof = on != 0;
    return FDTD_OK;
}

fdtd_status fdtd_get_timings(fdtd_handle h, fdtd_timings* out)
{
    if (fdtd_status s = check_handle(h, true)) return s;
    if (!out) return FDTD_ERR_ARG;
    fdtd_timings t = h->tim;
    t.fused_step = h->impl && h->impl->has_interior() ? 1 : 0;
    t.paired_shell = h->impl && h->impl->paired_shell() ? 1 : 0;
    t.pdl_graphs = h->impl && h->impl->pdl_graphs() ? 1 : 0;
    t.paired_design = h->impl && h->impl->paired_design() ? 1 : 0;
    const double ts = h->d.precision == 64 ? 8.0 : 4.0;
    // algorithmic bytes per launch: every state word read once and written once
    const double nc = (double)h->ncell, nd = (double)h->nd, nod = (double)(h->nd - h->ngap);
    // interior (fused) kernel: E^n and H read, H written, E written outside the design box;
    // shell kernels: H: E^n, H read, H written; E: H, E^n read, E written (outside the design box);
    // psi: per CPML slab cell and axis two psi_H read and written (H update), two psi_E (E update), in
    // the kernel that owns the cell
    double bst = 0.0, bsh = 0.0, bse = 0.0;
    const int n[3] = {h->d.nx, h->d.ny, h->d.nz};
    int ib[6] = {0, 0, 0, 0, 0, 0};
    if (h->impl) h->impl->interior_box(ib);
    for (int a = 0; a < 3; ++a) {
        const int lo = h->d.cpml[2 * a], hi = h->d.cpml[2 * a + 1];
        const double slab = (double)h->ncell / n[a] * (lo + hi);
        double in = (double)(std::max(0, std::min(ib[2 * a + 1], lo) - ib[2 * a]) +
                             std::max(0, ib[2 * a + 1] - std::max(ib[2 * a], n[a] - hi)));
        for (int b = 0; b < 3; ++b)
            if (b != a) in *= ib[2 * b + 1] - ib[2 * b];
        bst += 8.0 * ts * in;
        bsh += 4.0 * ts * (slab - in);
        bse += 4.0 * ts * (slab - in);
    }
    if (h->impl) {
        const double ni = (double)(ib[1] - ib[0]) * (ib[3] - ib[2]) * (ib[5] - ib[4]);
        const int* db = h->d.design_box;
        double ndi = 1.0;
        for (int a = 0; a < 3; ++a)
            ndi *= std::max(0, std::min(ib[2 * a + 1], db[2 * a + 1]) - std::max(ib[2 * a], db[2 * a]));
        if (box_count(db) == 0) ndi = 0.0;
        bst += 12.0 * ts * ni - 3.0 * ts * ndi;
        t.interior_cells = ni;
        t.interior_design_cells = ndi;
        bsh += 9.0 * ts * (nc - ni);
        bse += 9.0 * ts * ((nc - ni) - (nd - ndi));
    }
    double bd = 9.0 * ts * nd;                          // inside the design box: E^n, H^{n+1/2} read, E written
    if (h->impl) {
        int P = 0;
        if (h->d.precision == 64) {
            for (int k = 0; k < 3; ++k) P += as<double>(h)->ptot[k];
        } else {
            for (int k = 0; k < 3; ++k) P += as<float>(h)->ptot[k];
        }
        bd += nod * ts + nod * P * 2.0 * 2.0 * ts;      // rho read, Q r/w (design, non-gap)
        bd += nd * 3.0 * ts;                            // E snapshot write
        const double K = std::min(h->d.n_steps, kGraphSteps);
        t.dft_steps_per_launch = K;
        t.bytes_dft_per_launch = nd * (K * 3.0 * ts + 3.0 * h->d.n_freq * 16.0 * 2.0);  // snapshots + FP64 acc r/w
        t.bytes_grad_per_launch = nd * (2.0 * 3.0 * h->d.n_freq * 16.0 + ts + 8.0);     // both DFTs, rho, grad
    }
    t.bytes_shell_h_per_launch = bsh;
    t.bytes_step_per_launch = bst;
    t.bytes_shell_e_per_launch = bse;
    t.bytes_ed_per_launch = bd;
    *out = t;
    return FDTD_OK;
}

fdtd_status fdtd_reset_timings(fdtd_handle h)
{
    if (fdtd_status s = check_handle(h, true)) return s;
    h->tim = fdtd_timings{};
    return FDTD_OK;
}

fdtd_status fdtd_get_info(fdtd_handle h, double* dt, size_t* n_design, size_t* n_gap, size_t* device_bytes)
{
    if (fdtd_status s = check_handle(h, true)) return s;
    if (dt) *dt = h->dt;
    if (n_design) *n_design = h->nvar;
    if (n_gap) *n_gap = h->ngap;
    if (device_bytes) *device_bytes = h->bytes;
    return FDTD_OK;
}

fdtd_status fdtd_cancel(fdtd_handle h)
{
    if (!h) return FDTD_ERR_ARG;
    h->cancel.store(1);
    return FDTD_OK;
}

const char* fdtd_last_error(fdtd_handle h) { return h ? h->err.c_str() : g_last_error.c_str(); }

fdtd_status fdtd_destroy(fdtd_handle h)
{
    if (!h) return FDTD_ERR_ARG;
    batch_detach(h);
    cudaSetDevice(h->device);
    if (h->work) cudaStreamSynchronize(h->work);
    h->impl.reset();
    if (h->work) {
        h->free_all();
        cudaStreamSynchronize(h->work);
    }
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    if (h->fence) cudaEventDestroy(h->fence);
    if (h->bfence) cudaEventDestroy(h->bfence);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->join) cudaEventDestroy(h->join);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->work) cudaStreamDestroy(h->work);
    delete h;
    return FDTD_OK;
}

}  // extern "C"
