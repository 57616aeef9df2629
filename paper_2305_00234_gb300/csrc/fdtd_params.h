// Parameter structs shared by the kernels (fdtd_kernels.cuh) and the host code (fdtd_api.cu).
#pragma once
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
#ifndef FDTD_PZ
#define FDTD_PZ 2
#endif
#ifndef FDTD_H_MINB
#define FDTD_H_MINB 6
#endif
#ifndef FDTD_EBG_MINB
#define FDTD_EBG_MINB 4
#endif
#ifndef FDTD_ED_MINB
#define FDTD_ED_MINB 4
#endif
constexpr int kPZ = FDTD_PZ;      // z planes per thread in the H and background E kernels

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
    T* E[3];
    T* H[3];
    T* psiE[3][2];               // component c, derivative axis (c+1+t)%3
    T* psiH[3][2];
    const T* pmlE[3];            // per axis, per slab index: {1/kappa, b, c, 0} at integer positions
    const T* pmlH[3];            //                           ... at half-integer positions
    T inv_dx, ch;                // 1/dx, dt/mu0
    T bg_ca[3], bg_cb[3];        // background: E' = ca E + cb drive
    T D1[3], dD[3], N1[3], dN[3], hg;   // design: D(rho) = D1 + rho dD + hg rho(1-rho), N likewise
    int P[3], P1[3];             // poles per component (m1 first, P1 of them)
    const PoleTable<T>* poles;
    const T* rho;                // design box density
    cpx<T>* Q[3];                // pole currents [P[c]][nd]
    int K;                       // snapshot ring length (steps per DFT block)
    T* snap;                     // E snapshots of the design box [K][3][nd]
    int nb;                      // point-source basis functions (0 = none)
    const T* src_r;              // [(local sample)*nb + q], local sample = local voxel*3 + c
    const T* src_wave;           // [n*nb + q]
    int tfsf_i0;                 // first total-field x index, -1 = no TF/SF
    const T* einc;               // E_inc^n at x = i0 dx
    const T* hinc;               // H_inc^{n+1/2} at x = (i0 - 1/2) dx
    int* ctl;                    // [0] step n, [1] finished blocks of the advancing launch, [2] flags
    unsigned nblocks_e;          // blocks of e_bg_kernel
    unsigned nblocks_d;          // blocks of e_design_kernel
    T blowup;
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
    double* grad64;              // one of grad64 / grad32 is non-null
    float* grad32;
    double* partial;             // [gridDim.x + 1]
    unsigned* counter;
};

}  // namespace fdtd
