// Device kernels of the CCPR time-domain adjoint gradient (arXiv 2305.00234) for sm_103a.
//
// One Yee time step is a background step (fdtd_step.cuh: H^{n+1/2} everywhere, Eq. (Maxwells)c, and
// E^{n+1} outside the design box, with CFS-CPML psi in the edge slabs, the TF/SF plane and point
// sources) and
//   e_design_kernel: E^{n+1} inside the design box: the conductivity and the CCPR pole currents of
//                    both materials weighted by 1-rho and rho (Eqs. (Maxwells)a,b, (eps_mixed),
//                    (sigma_mixed), (Poles_mixed)), the pole recursion
//                    Q <- Q + (alpha-1) Q + beta (E^{n+1}+E^n), and an E snapshot for the DFT;
// and, every kMaxSnap steps, dft_kernel: the running FP64 DFT over the design box.  The gradient
// kernel evaluates the structure of Eq. (Gradient_analytic) per voxel (or per E sample with the
// per-sample density layout) with a deterministic warp-shuffle reduction of its squared norm.
//
// Thread layout of the per-cell kernels: blocks of (32, 8) threads over (x, y); x is the fastest
// array axis, so each warp reads and writes 128 contiguous bytes per field (FP32).
//
// The step index n lives in device memory (ctl[0]) so that a captured CUDA graph of K steps can be
// replayed: every kernel reads it, and the last block of the E phase (the shell-E and design-E
// launches, counted together) advances it.
#pragma once
#include "fdtd_params.h"

namespace fdtd {

__device__ __forceinline__ bool in_box(const int* b, int i, int j, int k)
{
    return i >= b[0] && i < b[1] && j >= b[2] && j < b[3] && k >= b[4] && k < b[5];
}

// Index inside the two CPML slabs [0, lo) and [n-hi, n) of one axis, -1 outside.
__device__ __forceinline__ int slab_index(int l, int lo, int hi, int n)
{
    return l < lo ? l : (l >= n - hi ? lo + (l - (n - hi)) : -1);
}

template <typename T>
__device__ __forceinline__ long long psi_index(const KParams<T>& p, int i, int j, int k, int a, int s)
{
    if (a == 0) return ((long long)k * p.ny + j) * p.W[0] + s;
    if (a == 1) return ((long long)k * p.W[1] + s) * p.nx + i;
    return ((long long)s * p.ny + j) * p.nx + i;
}

// CFS-CPML: psi <- b psi + c d ; derivative -> d / kappa + psi.
#ifndef FDTD_PML4
#define FDTD_PML4 1
#endif
// {1/kappa, b, c} of slab index s from a table of 4 values per index (FP32: one 16-byte load with
// FDTD_PML4, the default)
template <typename T>
__device__ __forceinline__ void pml_coef(const T* __restrict__ tab, int s, T& kinv, T& b, T& c)
{
#if FDTD_PML4
    if constexpr (sizeof(T) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(tab) + s);
        kinv = v.x;
        b = v.y;
        c = v.z;
        return;
    }
#endif
    kinv = __ldg(tab + 4 * s);
    b = __ldg(tab + 4 * s + 1);
    c = __ldg(tab + 4 * s + 2);
}

template <typename T>
__device__ __forceinline__ T stretch(T d, const T* __restrict__ tab, int s, T* psi)
{
    T kinv, b, c;
    pml_coef(tab, s, kinv, b, c);
    const T v = b * (*psi) + c * d;
    *psi = v;
    return d * kinv + v;
}

template <typename T>
__device__ __forceinline__ T ldg_t(const T* p) { return __ldg(p); }

#ifndef FDTD_ED_FASTDIV
#define FDTD_ED_FASTDIV 1
#endif
// a / b of the design update: in FP32 (FDTD_ED_FASTDIV, default) the hardware reciprocal and a multiply,
// at most 2 ulp for normal b (D is a positive normal number here; measured 4% faster than the IEEE
// division); in FP64, and with FDTD_ED_FASTDIV 0, the IEEE division
__device__ __forceinline__ float div_t(float a, float b)
{
#if FDTD_ED_FASTDIV
    return __fdividef(a, b);
#else
    return a / b;
#endif
}
__device__ __forceinline__ double div_t(double a, double b) { return a / b; }

// Load of solver state (fields, psi, pole currents, density, snapshots, DFT accumulators).  CG: through
// L2 only, bypassing L1, for work items of a persistent kernel, where an earlier item on the same SM may
// have left lines in L1 that another SM has since rewritten.
template <bool CG, typename T>
__device__ __forceinline__ T ldf(const T* p)
{
    if constexpr (CG)
        return __ldcg(p);
    else
        return *p;
}
template <bool CG, typename T>
__device__ __forceinline__ cpx<T> ldf(const cpx<T>* p)
{
    using V = typename vec2_of<T>::type;
    const V v = ldf<CG>(reinterpret_cast<const V*>(p));
    return cpx<T>{v.x, v.y};
}

template <typename T>
__device__ __forceinline__ cpx<T> ldg_c(const cpx<T>* p)
{
    cpx<T> v;
    v.re = __ldg(&p->re);
    v.im = __ldg(&p->im);
    return v;
}

// E update of one design sample of component C (blended), with Q^n:
//   E' = (N(rho) E + drive - sum_p kappa_p Re{g_p Q_p}) / D(rho),
//   Q_p <- Q_p + (alpha_p - 1) Q_p + beta_p (E' + E).
// MP bounds the poles per component at compile time so the pole currents stay in registers;
// design_load fetches them, design_update updates E and stores them back.  The pole coefficients
// come in the kernel's parameter space (C and the pole index are compile-time, so they are
// constant-bank operands).
// dq (paper mode): sum_p dkappa_p/drho Re{Q_p^{n+1} - Q_p^n} of this sample (-1 for m1's poles,
// +1 for m2's), the pole term of Eq. (Gradient_FDTD).
template <typename T, int MP, int C, bool CG = false>
__device__ __forceinline__ void design_load(const KParams<T>& p, long long dv, cpx<T> (&q)[MP > 0 ? MP : 1])
{
    const int P = p.P[C];
    const cpx<T>* __restrict__ Q = p.Q[C];
#pragma unroll
    for (int pp = 0; pp < MP; ++pp)
        if (pp < P) q[pp] = ldf<CG>(Q + pp * p.nd + dv);
}

template <typename T, int MP, int C>
__device__ __forceinline__ T design_update(const KParams<T>& p, const PoleTable<T>& tab, T rho, long long dv,
                                           const cpx<T> (&q)[MP > 0 ? MP : 1], T e_old, T drive, T& dq)
{
    dq = T(0);
    const T one = T(1);
    const T gm = p.hg * rho * (one - rho);
    const T D = p.D1[C] + rho * p.dD[C] + gm;
    const T N = p.N1[C] + rho * p.dN[C] - gm;
    if (MP == 0) return div_t(N * e_old + drive, D);
    const int P = p.P[C], P1 = p.P1[C];
    cpx<T>* __restrict__ Q = p.Q[C];
    T sq = T(0);
#pragma unroll
    for (int pp = 0; pp < MP; ++pp) {
        if (pp < P) {
            const T kap = pp < P1 ? one - rho : rho;
            const cpx<T> g = tab.g[C][pp];
            sq += kap * (g.re * q[pp].re - g.im * q[pp].im);
        }
    }
    const T e_new = div_t(N * e_old + drive - sq, D);
    const T es = e_new + e_old;
#pragma unroll
    for (int pp = 0; pp < MP; ++pp) {
        if (pp < P) {
            const cpx<T> a = tab.am1[C][pp];
            const cpx<T> b = tab.beta[C][pp];
            cpx<T> v;
            v.re = q[pp].re + (a.re * q[pp].re - a.im * q[pp].im) + b.re * es;
            v.im = q[pp].im + (a.re * q[pp].im + a.im * q[pp].re) + b.im * es;
            Q[pp * p.nd + dv] = v;
            dq += (pp < P1 ? -(v.re - q[pp].re) : (v.re - q[pp].re));
        }
    }
    return e_new;
}

template <typename T>
__device__ __forceinline__ T point_drive(const KParams<T>& p, int i, int j, int k, int c, int n)
{
    const long long lv = ((long long)(k - p.sb[4]) * (p.sb[3] - p.sb[2]) + (j - p.sb[2])) * (p.sb[1] - p.sb[0]) + (i - p.sb[0]);
    if (p.src_direct) return __ldg(p.src_wave + (long long)n * p.nsamp + lv * 3 + c);
    const T* r = p.src_r + (lv * 3 + c) * p.nb;
    const T* w = p.src_wave + (long long)n * p.nb;
    T s = T(0);
    for (int q = 0; q < p.nb; ++q) s += __ldg(r + q) * __ldg(w + q);
    return s;
}

template <typename T>
__device__ __forceinline__ int read_step(const int* ctl) { return __ldcg(ctl); }

// Programmatic dependent launch.  In the step graphs the kernels of a phase depend on those of the phase
// before through programmatic edges: a kernel's blocks may be launched before its predecessors have
// finished; pdl_wait() blocks until every predecessor has completed and its memory is visible, and
// pdl_trigger() lets the successors' blocks be launched once every block of this kernel has issued it.
// Every kernel of the step graphs waits first and triggers right after, so the next phase's blocks are
// already resident when a phase drains.  Both are no-ops for an ordinary launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// The last block of the launch that owns the step advance moves the device step counter on.
__device__ __forceinline__ void finish_step(int* ctl, unsigned nblocks, int n)
{
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        __threadfence();
        const unsigned prev = atomicAdd((unsigned*)(ctl + 1), 1u);
        if (prev == nblocks - 1) {
            ctl[1] = 0;
            atomicExch(ctl, n + 1);
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------------------------
// E update inside the working box.  A thread owns one component c of the (x, y) column of a block
// of p.edz planes (blockIdx.z = 3 zc + c, so the three components of a plane run in neighbouring
// blocks and share its H in L2; the per-block set-up and step-advance bookkeeping are paid once per
// p.edz planes) and handles its planes kEdPZ at a time, every load of a batch (the pole currents
// included) before any store: blended CCPR update of the design samples, background
// update of the gap samples and of samples outside their component's sample box, point sources,
// the E snapshot for the blocked DFT and the paper-mode records.  The working box lies outside the
// CPML, so there is no psi here.  Owns the step advance.
template <typename T, int MP>
constexpr int ed_min_blocks()
{
#ifdef FDTD_ED_MINB
    return FDTD_ED_MINB;
#else
    return sizeof(T) == 8 ? (MP <= 4 ? 4 : (MP <= 8 ? 3 : 2)) : (MP <= 4 ? 5 : (MP <= 8 ? 4 : 3));
#endif
}

// L2 prefetch (no registers held) of a line a coming plane's update reads.
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
#ifndef FDTD_DFT_PF
#define FDTD_DFT_PF 1   // 1: dft_voxel prefetches its accumulators into L2 first (config 2: 0.243 -> 0.212 ms)
#endif
#ifndef FDTD_ED_PF
#define FDTD_ED_PF 0   // planes ahead in e_design_column (0: none)
#endif

// One component C of the (x, y) column (i, j), planes [k0, k1); returns max |E| of its samples.
template <typename T, int MP, int C, bool CG = false>
__device__ __forceinline__ T e_design_column(const KParams<T>& p, const PoleTable<T>& tab, int i, int j, int k0, int k1, int n)
{
    constexpr int PZ = kEdPZ;
    // (curl H)_C = (Ha - Ha(la - 1)) - (Hb - Hb(lb - 1)): C = 0: Hz along y, Hy along z;
    // C = 1: Hx along z, Hz along x; C = 2: Hy along x, Hx along y
    constexpr int ca = C == 0 ? 2 : C - 1, cb = C == 2 ? 0 : C + 1;
    const unsigned oa = C == 0 ? (unsigned)p.nx : (C == 1 ? (unsigned)p.plane : 1u);
    const unsigned ob = C == 0 ? (unsigned)p.plane : (C == 1 ? 1u : (unsigned)p.nx);
    const T* __restrict__ Ha = p.Hn[ca];   // H^{n+1/2}, just written by the H update
    const T* __restrict__ Hb = p.Hn[cb];
    const T* __restrict__ Ec = p.E[C];     // E^n
    const T* __restrict__ rc = p.rhoc[C];
    const unsigned plane = (unsigned)p.plane, col = (unsigned)j * (unsigned)p.nx + (unsigned)i;
    const long long dcol = (long long)(j - p.db[2]) * p.dnx + (i - p.db[0]);
    const bool inxy_m = i >= p.mb[C][0] && i < p.mb[C][1] && j >= p.mb[C][2] && j < p.mb[C][3];
    const bool inxy_g = i >= p.gb[0] && i < p.gb[1] && j >= p.gb[2] && j < p.gb[3];
    const long long slot0 = (long long)((n - p.snap0) % p.K) * 3 * p.nd + C * p.nd;
    const T hinc_n = (C == 2 && i == p.tfsf_i0) ? __ldg(p.hinc + n) * p.inv_dx : T(0);
    T emax = T(0);
    for (int kb = k0; kb < k1; kb += PZ) {
        T ha[PZ], ham[PZ], hb[PZ], hbm[PZ], e0[PZ], rho[PZ];
        cpx<T> q[PZ][MP > 0 ? MP : 1];
        bool ds[PZ];
#pragma unroll
        for (int r = 0; r < PZ; ++r) {
            const int k = kb + r;
            ds[r] = false;
            if (k >= k1) continue;
            const unsigned id = (unsigned)k * plane + col;
            const long long dv = (long long)(k - p.db[4]) * p.dplane + dcol;
            const int la = C == 0 ? j : (C == 1 ? k : i), lb = C == 0 ? k : (C == 1 ? i : j);
            ha[r] = ldf<CG>(Ha + id);
            hb[r] = ldf<CG>(Hb + id);
            ham[r] = la > 0 ? ldf<CG>(Ha + id - oa) : T(0);
            hbm[r] = lb > 0 ? ldf<CG>(Hb + id - ob) : T(0);
            if constexpr (!CG && FDTD_ED_PF > 0) {   // the rows of a coming plane into L2
                if (k + FDTD_ED_PF < k1) {
                    const unsigned ip = id + FDTD_ED_PF * plane;
                    const long long dp = dv + FDTD_ED_PF * p.dplane;
                    prefetch_l2(Ha + ip);
                    prefetch_l2(Hb + ip);
                    prefetch_l2(Ec + ip);
                    prefetch_l2(rc + dp);
#pragma unroll
                    for (int pp = 0; pp < (MP > 0 ? MP : 1); ++pp)
                        if (pp < p.P[C]) prefetch_l2(p.Q[C] + pp * p.nd + dp);
                }
            }
            e0[r] = ldf<CG>(Ec + id);
            ds[r] = inxy_m && k >= p.mb[C][4] && k < p.mb[C][5] && !(inxy_g && k >= p.gb[4] && k < p.gb[5]);
            rho[r] = ds[r] ? ldf<CG>(rc + dv) : T(0);
            if (ds[r]) design_load<T, MP, C, CG>(p, dv, q[r]);
        }
#pragma unroll
        for (int r = 0; r < PZ; ++r) {
            const int k = kb + r;
            if (k >= k1) continue;
            const unsigned id = (unsigned)k * plane + col;
            const long long dv = (long long)(k - p.db[4]) * p.dplane + dcol;
            const int la = C == 0 ? j : (C == 1 ? k : i), lb = C == 0 ? k : (C == 1 ? i : j);
            T d = ((ha[r] - ham[r]) - (hb[r] - hbm[r])) * p.inv_dx - hinc_n;
            if (p.nb > 0 && in_box(p.sb, i, j, k)) d += point_drive(p, i, j, k, C, n);
            T dq = T(0);
            T e = ds[r] ? design_update<T, MP, C>(p, tab, rho[r], dv, q[r], e0[r], d, dq) : p.bg_ca[C] * e0[r] + p.bg_cb[C] * d;
            if (!(la > 0 && lb > 0)) e = e0[r];   // PEC walls: components tangential to a wall at index 0 stay zero
            p.En[C][id] = e;
            const long long slot = slot0 + dv;
            p.snap[slot] = e;
            if (p.hist_dq) p.hist_dq[slot] = dq;   // paper mode, recompute pass
            if (p.td_acc && inxy_g && k >= p.gb[4] && k < p.gb[5]) {   // paper mode, forward pass: gap samples
                const long long lg = (((long long)(k - p.gb[4]) * p.gny + (j - p.gb[2])) * p.gnx + (i - p.gb[0])) * 3 + C;
                p.td_acc[lg] += (double)e * (double)e;
                p.gap_hist[(long long)n * p.nsamp + lg] = e;
            }
            emax = fmax(emax, fabs(e));
        }
    }
    return emax;
}

template <typename T, int MP>
__global__ void __launch_bounds__(kBX * kBY, ed_min_blocks<T, MP>()) e_design_kernel(const KParams<T> p, const PoleTable<T> tab)
{
    const int zc = blockIdx.z / 3, c = blockIdx.z - 3 * zc;
    int i, j;
    if (FDTD_ED_FLAT) {   // columns in row order, kBX * kBY per block
        const int dnx = p.db[1] - p.db[0];
        const int col = blockIdx.x * (kBX * kBY) + threadIdx.y * kBX + threadIdx.x;
        const int y = col / dnx;
        i = p.db[0] + (col - y * dnx);
        j = p.db[2] + y;
    } else {
        i = p.db[0] + blockIdx.x * kBX + threadIdx.x;
        j = p.db[2] + blockIdx.y * kBY + threadIdx.y;
    }
    const int k0 = p.db[4] + zc * p.edz, k1 = min(p.db[5], k0 + p.edz);
    pdl_wait();
    pdl_trigger();
    const int n = read_step<T>(p.ctl);
    if (i < p.db[1] && j < p.db[3]) {
        const T emax = c == 0 ? e_design_column<T, MP, 0>(p, tab, i, j, k0, k1, n)
                     : c == 1 ? e_design_column<T, MP, 1>(p, tab, i, j, k0, k1, n)
                              : e_design_column<T, MP, 2>(p, tab, i, j, k0, k1, n);
        if (!(emax < p.blowup)) atomicOr(p.ctl + 2, 1);
    }
    finish_step(p.ctl, p.nblocks_e, n);
}

// ---------------------------------------------------------------------------------------------
// Blocked running DFT over the design box.  After cnt steps n0..n0+cnt-1 (n0 = ctl[0] - cnt), each
// thread owns one design voxel: it reads the cnt snapshots E^{n+1} of its three samples, forms the
// block sums sum_s E^{n0+s+1} (cos, -sin)(w_f (n0+s+1) dt) in the accumulation type A, and adds
// them to the FP64 accumulators, which are read and written once per block instead of every step.
// ---------------------------------------------------------------------------------------------
// The fold of one voxel v: steps n0 .. n0 + cnt - 1 (cnt <= kMaxSnap).
template <typename T, bool CG>
__device__ __forceinline__ void dft_voxel(const DParams<T>& d, long long v, int n0, int cnt)
{
#if FDTD_DFT_PF
    if constexpr (!CG)   // the FP64 accumulators into L2 while the snapshots load
        for (int q = 0; q < 3 * d.nf; ++q) prefetch_l2(d.dft + (long long)q * d.nd + v);
#endif
    T e[kMaxSnap][3];
#pragma unroll
    for (int s = 0; s < kMaxSnap; ++s) {
        if (s < cnt) {
            const T* sp = d.snap + (long long)((n0 + s) % d.K) * 3 * d.nd + v;
            e[s][0] = ldf<CG>(sp);
            e[s][1] = ldf<CG>(sp + d.nd);
            e[s][2] = ldf<CG>(sp + 2 * d.nd);
        }
    }
    for (int f = 0; f < d.nf; ++f) {
        T re[3] = {T(0), T(0), T(0)}, im[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int s = 0; s < kMaxSnap; ++s) {
            if (s < cnt) {
                const auto ph = __ldg(d.ph + (long long)(n0 + s + 1) * d.nf + f);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    re[c] = fma(e[s][c], ph.x, re[c]);
                    im[c] = fma(-e[s][c], ph.y, im[c]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double2* acc = d.dft + (long long)(f * 3 + c) * d.nd + v;
            double2 a = ldf<CG>(acc);
            a.x += (double)re[c];
            a.y += (double)im[c];
            *acc = a;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kReduceThreads) dft_kernel(const DParams<T> d, int cnt)
{
    pdl_wait();                                   // the snapshots of the block's last step
    pdl_trigger();
    const long long v = (long long)blockIdx.x * kReduceThreads + threadIdx.x;
    if (v >= d.nd) return;
    dft_voxel<T, false>(d, v, __ldcg(d.ctl) - cnt, cnt);
}

// ---------------------------------------------------------------------------------------------
// Gradient: per design voxel v (not gap),
//   G_v = -sum_c sum_f 2 Re{ (A_cf + (1 - 2 rho_v) B_cf) Ehat_cf,v Lambda_cf,v },
// A_cf = dY/drho without the gamma term, B_cf = gamma (z+1)/2 (host-precomputed, FP64).
// The squared norm is reduced per block with warp shuffles into partial[blockIdx.x]; the last
// block adds the partials in block order (deterministic) into partial[gridDim.x].
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__global__ void __launch_bounds__(kReduceThreads) grad_kernel(const GParams<T> g)
{
    __shared__ double warp_part[kReduceThreads / 32];
    __shared__ bool last;
    const long long q = (long long)blockIdx.x * kReduceThreads + threadIdx.x;
    double G = 0.0;
    if (q < (g.per_comp ? g.nout : g.nd)) {
        // per voxel: v = q, the three owned samples share rho; per sample: one component c
        long long v = q;
        int c0 = 0, c1 = 3;
        if (g.per_comp) {
            c0 = q >= g.off[2] ? 2 : (q >= g.off[1] ? 1 : 0);
            c1 = c0 + 1;
            const long long l = q - g.off[c0];
            const int mx = g.mdim[c0][0], my = g.mdim[c0][1];
            v = ((l / ((long long)mx * my)) * g.dny + (l / mx) % my) * g.dnx + l % mx;
        }
        const int i = g.db[0] + (int)(v % g.dnx);
        const int j = g.db[2] + (int)((v / g.dnx) % g.dny);
        const int k = g.db[4] + (int)(v / ((long long)g.dnx * g.dny));
        if (!in_box(g.gb, i, j, k)) {
            for (int c = c0; c < c1; ++c) {
                const double s = 1.0 - 2.0 * (double)(g.per_comp ? g.rhoc[c][v] : g.rho[v]);
                for (int f = 0; f < g.nf; ++f) {
                    const double2 A = __ldg(g.AB + (c * g.nf + f) * 2);
                    const double2 B = __ldg(g.AB + (c * g.nf + f) * 2 + 1);
                    const double dyr = A.x + s * B.x, dyi = A.y + s * B.y;
                    const long long o = (long long)(f * 3 + c) * g.nd + v;
                    const double2 e = g.dft_f[o], l = g.dft_a[o];
                    const double eli_r = e.x * l.x - e.y * l.y, eli_i = e.x * l.y + e.y * l.x;
                    G -= 2.0 * (dyr * eli_r - dyi * eli_i);
                }
            }
        }
        if (g.grad64) g.grad64[q] = G;
        if (g.grad32) g.grad32[q] = (float)G;
    }
    double s2 = warp_sum(G * G);
    if ((threadIdx.x & 31) == 0) warp_part[threadIdx.x >> 5] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < kReduceThreads / 32; ++w) b += warp_part[w];
        g.partial[blockIdx.x] = b;
        __threadfence();
        last = (atomicAdd(g.counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double t = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) t += ((volatile double*)g.partial)[b];
        g.partial[gridDim.x] = t;
        *g.counter = 0;
    }
}


// Per-sample density (compact: component c's samples (z, y, x) over extents md[c], components
// concatenated) -> dst[c][dv] over the working box (dnx, dny); values checked to lie in [0, 1].
template <typename T, typename S>
__global__ void rho_scatter_kernel(const S* __restrict__ src, long long n, long long o1, long long o2, int3 m0, int3 m1,
                                   int3 m2, int dnx, int dny, long long nd, T* __restrict__ dst, int* flag)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int c = q >= o2 ? 2 : (q >= o1 ? 1 : 0);
    const int3 md = c == 0 ? m0 : (c == 1 ? m1 : m2);
    const long long l = q - (c == 0 ? 0 : (c == 1 ? o1 : o2));
    const long long dv = ((l / ((long long)md.x * md.y)) * dny + (l / md.x) % md.y) * dnx + l % md.x;
    const S r = src[q];
    if (!(r >= S(0) && r <= S(1))) atomicOr(flag, 2);
    dst[c * nd + dv] = (T)r;
}

// ---------------------------------------------------------------------------------------------
// Paper mode (time-domain objective of Eq. (Objective_analyitically_enhancement) and gradient
// Eq. (Gradient_FDTD) with checkpoint-recompute).
// ---------------------------------------------------------------------------------------------
// E of the current state at every design-box sample -> out[c][dv] (a history slot).
template <typename T>
__global__ void gather_design_e_kernel(const KParams<T> p, T* __restrict__ out)
{
    const long long dv = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (dv >= p.nd) return;
    const int i = p.db[0] + (int)(dv % p.dnx), j = p.db[2] + (int)((dv / p.dnx) % p.dny), k = p.db[4] + (int)(dv / p.dplane);
    const long long id = ((long long)k * p.ny + j) * p.nx + i;
    out[dv] = p.E[0][id];
    out[p.nd + dv] = p.E[1][id];
    out[2 * p.nd + dv] = p.E[2][id];
}

// Adjoint drive of SI Eq. (AdjointSystem): the time-reversed functional derivative eps0 E at every
// gap sample, delayed one step: drive[m][s] = eps0 E_s^{M-m-1}, E^{n+1} = gh[n][s], E^0 = 0.
template <typename T>
__global__ void paper_drive_kernel(const T* __restrict__ gh, T* __restrict__ drive, int M, int ns, double eps0)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long long)M * ns) return;
    const int m = (int)(q / ns), s = (int)(q % ns);
    const int n = M - m - 2;
    drive[q] = n >= 0 ? (T)(eps0 * (double)gh[(long long)n * ns + s]) : T(0);
}

// One segment of Eq. (Gradient_FDTD) per design voxel: adjoint levels m = a0+1..a0+len pair with
// forward levels L = M - m = n0+len-1..n0 (slot len - q for q = m - a0):
//   g += sum_c [ -eps0 deps_c E^L (Et^m - Et^{m-1}) - (dsig_c + (1-2 rho) gamma) dt E^L (Et^m + Et^{m-1})/2
//                + 2 sum_p dkappa_p Re{Q^L - Q^{L+1}} w ],   w = (Et^m + Et^{m-1})/2 or Et^{m-1};
// sum_p dkappa_p Re{Q^L - Q^{L+1}} = -dq[L].  Gap voxels are skipped (gradient 0).
template <typename T>
__global__ void paper_grad_kernel(const PParams<T> g)
{
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.nd) return;
    const int i = g.db[0] + (int)(v % g.dnx), j = g.db[2] + (int)((v / g.dnx) % g.dny);
    const int k = g.db[4] + (int)(v / ((long long)g.dnx * g.dny));
    if (i >= g.gb[0] && i < g.gb[1] && j >= g.gb[2] && j < g.gb[3] && k >= g.gb[4] && k < g.gb[5]) return;
    const double rho = (double)g.rho[v];
    const long long st = 3 * g.nd;
    double acc = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double a1 = -g.eps0 * g.deps[c], a2 = -(g.dsig[c] + (1.0 - 2.0 * rho) * g.gamma) * g.dt;
        double t = 0.0;
        double am = (double)g.ha[c * g.nd + v];               // Et^{a0}
        for (int q = 1; q <= g.len; ++q) {
            const double ap = (double)g.ha[q * st + c * g.nd + v];
            const double e = (double)g.he[(g.len - q) * st + c * g.nd + v];
            const double dq = (double)g.hq[(g.len - q) * st + c * g.nd + v];
            const double avg = 0.5 * (ap + am);
            t += a1 * e * (ap - am) + a2 * e * avg - 2.0 * dq * (g.single ? am : avg);
            am = ap;
        }
        acc += t;
    }
    g.gsum[v] += acc;
}

}  // namespace fdtd
