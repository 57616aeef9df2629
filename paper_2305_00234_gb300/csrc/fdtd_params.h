// Parameter structs shared by the kernels (fdtd_kernels.cuh) and the host code (fdtd_api.cu).
#pragma once
#include <cuda.h>            // CUtensorMap (type only; the encoder is fetched at run time)
#include <cuda_runtime.h>
#include <stdint.h>

namespace fdtd {


constexpr int kMaxPoles = 16;     // per component, m1 + m2
constexpr int kMaxFreq = 8;
constexpr int kMaxBasis = 2 * kMaxFreq;
constexpr int kBX = 32;
constexpr int kBY = 8;
constexpr int kReduceThreads = 256;
constexpr int kMaxSnap = 16;      // steps per blocked DFT update (snapshot ring length)
#ifndef FDTD_SHELL_PZ
#define FDTD_SHELL_PZ 2
#endif
#ifndef FDTD_SHELL_MINB
#define FDTD_SHELL_MINB 4
#endif
#ifndef FDTD_KC
#define FDTD_KC 8
#endif
#ifndef FDTD_SHELL_KZ
#define FDTD_SHELL_KZ 8
#endif
#ifndef FDTD_ED_Z
#define FDTD_ED_Z 8
#endif
#ifndef FDTD_ED_PZ
#define FDTD_ED_PZ 1
#endif
constexpr int kEdZ = FDTD_ED_Z;     // most z planes per thread in the design-E kernel
constexpr int kEdPZ = FDTD_ED_PZ;   // of which loaded per batch
// FDTD_ED_FLAT 1 (default): the one-sample design-E kernel takes (x, y) columns 256 at a time in row order
// (every lane busy on working boxes narrower than 32 cells: the paper grid's 26-cell-deep box, design E
// 0.0220 -> 0.0213 ms); 0: 32 x 8 column tiles
#ifndef FDTD_ED_FLAT
#define FDTD_ED_FLAT 1
#endif
constexpr int kShellPZ = FDTD_SHELL_PZ;   // z planes per batch of loads in the shell kernels
constexpr int kShellKZ = FDTD_SHELL_KZ;   // most z planes per thread in the shell kernels (a multiple of kShellPZ)
constexpr int kKC = FDTD_KC;      // z planes per block of the fused step kernel

// Fused step kernel tile: kTX x kTY cells of one z plane, kTX/2 x kTY threads, each thread two
// x-adjacent cells.  Boxes staged by TMA per plane: x in [i0 - kOX, i0 - kOX + kSX) (a start that is a
// multiple of 4 elements, so 16-byte aligned for 4- and 8-byte types), E rows [j0 - 1, j0 + kTY],
// H rows [j0 - 1, j0 + kTY - 1], all three components.
constexpr int kTX = 32;
constexpr int kTY = 16;
constexpr int kPX = kTX / 2;
constexpr int kOX = 4;
constexpr int kSX = kTX + 8;
constexpr int kSYE = kTY + 2;
constexpr int kSYH = kTY + 1;
constexpr int kHW = kTX + 2;      // row of the new-H tile: [1] is x = i0 - 1, [2 + xr] is x = i0 + xr

__host__ __device__ constexpr size_t align128(size_t b) { return (b + 127) / 128 * 128; }

#ifndef FDTD_STEP_NE
#define FDTD_STEP_NE 4
#endif
#ifndef FDTD_STEP_NH
#define FDTD_STEP_NH 3
#endif
#ifndef FDTD_STEP_MINB
#define FDTD_STEP_MINB 3
#endif
template <typename T>
struct StepCfg;
template <>
struct StepCfg<float> {   // E / H ring slots, resident blocks per SM
    static constexpr int NE = FDTD_STEP_NE, NH = FDTD_STEP_NH, MINB = FDTD_STEP_MINB;
};
template <>
struct StepCfg<double> {
    static constexpr int NE = 3, NH = 2, MINB = 2;
};
template <typename T>
struct StepSmem {
    static constexpr unsigned e_tx = 3u * kSYE * kSX * sizeof(T);    // bytes one E plane load delivers
    static constexpr unsigned h_tx = 3u * kSYH * kSX * sizeof(T);
    static constexpr size_t e_slot = align128(e_tx);
    static constexpr size_t h_slot = align128(h_tx);
    static constexpr size_t h_new = align128(2 * 3 * (size_t)kSYH * kHW * sizeof(T));   // two tiles
    static constexpr size_t table = 128;                                                // per-plane path
    static constexpr size_t bars = 128;
    static constexpr size_t total = StepCfg<T>::NE * e_slot + StepCfg<T>::NH * h_slot + h_new + table + bars + 128;
};

// The cells outside the interior box, as at most six boxes, for the shell kernels: block b of a
// launch belongs to the box q with first[q] <= b < first[q + 1].
struct ShellBoxes {
    int n;
    int b[6][6];          // half-open x0, x1, y0, y1, z0, z1
    unsigned first[7];
    int kz;               // z planes per thread (<= kShellKZ)
    int pair;             // 1: the paired kernels (a thread per two x-adjacent columns; every x bound even)
};

// Tensor maps of the buffers one step reads: E^n and H^{n-1/2}, each 4-D (x, y, z, component).
struct StepMaps {   // (CUtensorMap is 64-byte aligned)
    CUtensorMap e, h;
};

template <typename T>
struct cpx {
    T re, im;
};

// Pole coefficients of one handle, in device memory (uniform loads through the read-only path).
template <typename T>
struct PoleTable {
    cpx<T> am1[3][kMaxPoles];    // alpha - 1 = e^{a dt} - 1
    cpx<T> beta[3][kMaxPoles];   // eps0 c (e^{a dt} - 1) / (2 a)
    cpx<T> g[3][kMaxPoles];      // (2/dt)(alpha - 1): weight of Re{(alpha-1) Q} in the E update
};

template <typename T>
struct KParams {
    int nx, ny, nz;
    long long plane, ncell;
    int db[6], gb[6], sb[6];     // design, gap, point-source boxes (half-open)
    int dnx, dny;
    long long dplane, nd;
    int gnx, gny;
    long long gplane;
    int cpl[3], cph[3], W[3];    // CPML thickness low / high, slab width per axis
    T* E[3];                     // E^n (read)
    T* H[3];                     // H^{n-1/2} (read)
    T* En[3];                    // E^{n+1} (written; the other buffer of the pair)
    T* Hn[3];                    // H^{n+1/2} (written)
    T* psiE[3][2];               // component c, derivative axis (c+1+t)%3; updated in place
    T* psiH[3][2];               // psi of the H update at n-1/2 (read)
    T* psiHn[3][2];              // ... at n+1/2 (written)
    const T* pmlE[3];            // per axis, per slab index: {1/kappa, b, c, 0} at integer positions
    const T* pmlH[3];            //                           ... at half-integer positions
    T inv_dx, ch;                // 1/dx, dt/mu0
    T bg_ca[3], bg_cb[3];        // background: E' = ca E + cb drive
    T bg_cbi[3];                 // cb / dx
    T D1[3], dD[3], N1[3], dN[3], hg;   // design: D(rho) = D1 + rho dD + hg rho(1-rho), N likewise
    int P[3], P1[3];             // poles per component (m1 first, P1 of them)
    const PoleTable<T>* poles;
    const T* rho;                // design box density
    // per-component design samples: E_c of voxel v is blended with density rhoc[c][v] when the
    // voxel lies in mb[c] and not in the gap (one density per voxel: rhoc[c] = rho, mb[c] = db)
    const T* rhoc[3];
    int mb[3][6];
    cpx<T>* Q[3];                // pole currents [P[c]][nd]
    int K;                       // snapshot ring length (steps per DFT block)
    int snap0;                   // step n writes its E^{n+1} snapshot to slot (n - snap0) mod K
    T* snap;                     // E snapshots of the design box [K][3][nd]
    int nb;                      // point-source basis functions (0 = none)
    int src_direct;              // 1: the drive of source-box sample s at step n is src_wave[n * nsamp + s]
    int nsamp;                   //    (s = local voxel * 3 + component), no basis expansion
    // time-domain (paper-mode) recording, all null otherwise
    double* td_acc;              // per gap sample (local voxel * 3 + c): sum over steps of (E^{n+1})^2
    T* gap_hist;                 // [n][local gap voxel * 3 + c]: E^{n+1} of the gap samples
    T* hist_dq;                  // [(n - snap0) mod K][3][nd]: sum_p dkappa_p/drho Re{Q_p^{n+1} - Q_p^n}
    const T* src_r;              // [(local sample)*nb + q], local sample = local voxel*3 + c
    const T* src_wave;           // [n*nb + q]
    int tfsf_i0;                 // first total-field x index, -1 = no TF/SF
    const T* einc;               // E_inc^n at x = i0 dx
    const T* hinc;               // H_inc^{n+1/2} at x = (i0 - 1/2) dx
    int n_steps;                 // steps of a run
    int* ctl;                    // [0] step n, [1] finished blocks of the advancing launch, [2] flags
    int ib[6];                   // interior box of the fused step kernel (empty: x0 = x1)
    unsigned nblocks_s;          // blocks of the background-E shell kernel
    unsigned nblocks_d;          // blocks of e_design_kernel
    int edz;                     // z planes per thread of e_design_kernel (<= kEdZ)
    int kc;                      // z planes per block of step_kernel (<= kKC)
    int ed_pair;                 // 1: e_design2_kernel (FP32, x-adjacent sample pairs; nx and the working box's
                                 // x origin and extent even, one density per voxel)
    unsigned nblocks_e;          // blocks of the E phase (shell E + design E); the last one advances the step
    T blowup;
    long long stall_ns;          // failure-path test hook (step_kernel): > 0 makes block (0, 0, 0) at step 0 wait
                                 // this long on an mbarrier that nothing completes; 0 = off
};

template <typename T>
struct vec2_of;
template <>
struct vec2_of<float> {
    using type = float2;
};
template <>
struct vec2_of<double> {
    using type = double2;
};

template <typename T>
struct DParams {
    long long nd;
    int nf, K;
    const T* snap;                          // [K][3][nd]
    double2* dft;                           // [nf][3][nd]
    const typename vec2_of<T>::type* ph;    // (cos, sin)(w_f n dt) in T, [(M+1)][nf]
    const int* ctl;
};

template <typename T>
struct GParams {
    int db[6], gb[6];
    int dnx, dny;
    long long nd;
    int nf;
    const double2* dft_f;
    const double2* dft_a;
    const double2* AB;           // [c][f][2]: A, B
    const T* rho;
    // per-sample layout (per_comp = 1): output q in [0, nout) is sample q - off[c] of component c,
    // (z, y, x) over extents mdim[c]; its density rhoc[c][dv] with dv its working-box voxel
    int per_comp;
    long long nout, off[4];
    int mdim[3][3];
    const T* rhoc[3];
    double* grad64;              // one of grad64 / grad32 is non-null
    float* grad32;
    double* partial;             // [gridDim.x + 1]
    unsigned* counter;
};

// ---- batched runs: one persistent launch advances several runs (different grids) together ----------
#ifndef FDTD_BATCH_MINB
#define FDTD_BATCH_MINB 2
#endif
constexpr int kMaxBatch = 16;          // runs of one launch
#ifndef FDTD_BATCH_THREADS
#define FDTD_BATCH_THREADS 256
#endif
constexpr int kBatchThreads = FDTD_BATCH_THREADS;   // threads of a block of the persistent kernel
constexpr int kMinBatchSZ = 4;         // z planes of a work item: 4 or 8 (<= kShellKZ) by grid size
constexpr int kMaxBatchSlabs = 65536 / kMinBatchSZ + 1;
static_assert(2 * kMinBatchSZ <= kShellKZ, "work items of up to kShellKZ planes");

// One run of the batch, device-resident.
template <typename T>
struct BatchSlot {
    KParams<T> kp[2];                  // the run's step parameters for even / odd steps
    DParams<T> dp;                     // its running DFT (forward or adjoint accumulators)
    unsigned* prog;                    // [nslab]: work items of the slab completed since the run started
    int nslab, nxyc;                   // slabs of sz planes x chunks of cw (x, y) columns
    int sz, cw;                        // work-item shape of this run
    int n0;                            // first step of the current launch
};

// One launch: run j (in order of phases, descending) takes phases 0 .. nph[j]-1 of this launch, 2 per step
// (H, E).  Work items are numbered round by round: round g holds phase g of every run with nph > g,
// run by run, each run's items slab-major.  Segment q covers rounds [seg_g0[q], seg_g0[q+1]) in which the
// first seg_m[q] runs take part; seg_t0[q] is its first item, seg_t0[nseg] the launch's item count.
struct BatchLaunch {
    int nruns, nseg;
    int slot[kMaxBatch];               // slot of run j in the device table
    long long pre[kMaxBatch + 1];      // items of one phase of runs 0 .. j-1
    int seg_g0[kMaxBatch + 1];
    int seg_m[kMaxBatch];
    long long seg_t0[kMaxBatch + 1];
    void* slots;                       // BatchSlot<T>[kMaxBatch]
    unsigned long long* ticket;        // next work item (zeroed before every launch)
    int* err;                          // [0]: 1 when a dependency wait gave up; [1]: the item that gave up
    const int* gate;                   // test hook: non-null makes item 0 also wait for *gate != 0
    unsigned long long wait_ns;        // limit of one dependency wait
};

// Paper-mode gradient, one checkpoint segment of forward levels n0..n0+len and adjoint levels
// a0..a0+len (a0 = M - n0 - len): Eq. (Gradient_FDTD) accumulated per design voxel.
template <typename T>
struct PParams {
    long long nd;
    int dnx, dny;
    int db[6], gb[6];
    const T* he;        // [len+1][3][nd] forward E, levels n0..n0+len
    const T* ha;        // [len+1][3][nd] adjoint E, levels a0..a0+len
    const T* hq;        // [len][3][nd] dq of forward steps n0..n0+len-1
    const T* rho;
    double* gsum;       // per design voxel, accumulated over segments
    int len;
    int single;         // pole term: 1 pairs the Q difference with one adjoint level, 0 the average of two
    double deps[3], dsig[3], gamma, eps0, dt;
};

}  // namespace fdtd
