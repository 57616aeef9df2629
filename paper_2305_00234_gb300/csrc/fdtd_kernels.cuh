// Device kernels of the CCPR time-domain adjoint gradient (arXiv 2305.00234) for sm_103a.
//
// One Yee time step is a background step (fdtd_step.cuh: H^{n+1/2} everywhere, Eq. (Maxwells)c, and
// E^{n+1} outside the design box, with CFS-CPML psi in the edge slabs, the TF/SF plane and point
// sources), then
//   e_design_kernel: E^{n+1} inside the design box: the conductivity and the CCPR pole currents of
//                    both materials weighted by 1-rho and rho (Eqs. (Maxwells)a,b, (eps_mixed),
//                    (sigma_mixed), (Poles_mixed)), the pole recursion
//                    Q <- Q + (alpha-1) Q + beta (E^{n+1}+E^n), and an E snapshot for the DFT;
// and, every kMaxSnap steps, dft_kernel: the running FP64 DFT over the design box.  The gradient
// kernel evaluates the structure of Eq. (Gradient_analytic) per voxel with a deterministic
// warp-shuffle reduction of its squared norm.
//
// Thread layout of the per-cell kernels: block (32, 8) over (x, y); x is the fastest array axis, so
// each warp reads and writes 128 contiguous bytes per field (FP32).
//
// The step index n lives in device memory (ctl[0]) so that a captured CUDA graph of K steps can be
// replayed: every kernel reads it, and the last block of e_design_kernel (of the background-E shell
// kernel when there is no design box) advances it.
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
template <typename T>
__device__ __forceinline__ T stretch(T d, const T* __restrict__ tab, int s, T* psi)
{
    const T kinv = __ldg(tab + 4 * s), b = __ldg(tab + 4 * s + 1), c = __ldg(tab + 4 * s + 2);
    const T v = b * (*psi) + c * d;
    *psi = v;
    return d * kinv + v;
}

template <typename T>
__device__ __forceinline__ T ldg_t(const T* p) { return __ldg(p); }

template <typename T>
__device__ __forceinline__ cpx<T> ldg_c(const cpx<T>* p)
{
    cpx<T> v;
    v.re = __ldg(&p->re);
    v.im = __ldg(&p->im);
    return v;
}

// E update of one design sample (blended), with Q^n:
//   E' = (N(rho) E + drive - sum_p kappa_p Re{g_p Q_p}) / D(rho),
//   Q_p <- Q_p + (alpha_p - 1) Q_p + beta_p (E' + E).
// MP bounds the poles per component at compile time so the pole currents stay in registers.
// dq (paper mode): sum_p dkappa_p/drho Re{Q_p^{n+1} - Q_p^n} of this sample (-1 for m1's poles,
// +1 for m2's), the pole term of Eq. (Gradient_FDTD).
template <typename T, int MP>
__device__ __forceinline__ T design_sample(const KParams<T>& p, int c, T rho, long long dv, T e_old, T drive, T& dq)
{
    dq = T(0);
    const T one = T(1);
    const T gm = p.hg * rho * (one - rho);
    const T D = p.D1[c] + rho * p.dD[c] + gm;
    const T N = p.N1[c] + rho * p.dN[c] - gm;
    if (MP == 0) return (N * e_old + drive) / D;
    const int P = p.P[c], P1 = p.P1[c];
    cpx<T>* __restrict__ Q = p.Q[c];
    const PoleTable<T>* __restrict__ tab = p.poles;
    cpx<T> q[MP > 0 ? MP : 1];
#pragma unroll
    for (int pp = 0; pp < MP; ++pp)
        if (pp < P) q[pp] = Q[pp * p.nd + dv];
    T sq = T(0);
#pragma unroll
    for (int pp = 0; pp < MP; ++pp) {
        if (pp < P) {
            const T kap = pp < P1 ? one - rho : rho;
            const cpx<T> g = ldg_c(&tab->g[c][pp]);
            sq += kap * (g.re * q[pp].re - g.im * q[pp].im);
        }
    }
    const T e_new = (N * e_old + drive - sq) / D;
    const T es = e_new + e_old;
#pragma unroll
    for (int pp = 0; pp < MP; ++pp) {
        if (pp < P) {
            const cpx<T> a = ldg_c(&tab->am1[c][pp]);
            const cpx<T> b = ldg_c(&tab->beta[c][pp]);
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
// E update inside the design box: blended CCPR update of the design voxels, background update of
// the gap voxels, point sources, and the E snapshot for the blocked DFT.  The design box lies
// outside the CPML, so there is no psi here.  One cell per thread; owns the step advance.
template <typename T, int MP>
__global__ void __launch_bounds__(kBX * kBY, FDTD_ED_MINB) e_design_kernel(const KParams<T> p)
{
    const int i = p.db[0] + blockIdx.x * kBX + threadIdx.x;
    const int j = p.db[2] + blockIdx.y * kBY + threadIdx.y;
    const int k = p.db[4] + blockIdx.z;
    const int n = read_step<T>(p.ctl);
    if (i < p.db[1] && j < p.db[3]) {
        const long long id = ((long long)k * p.ny + j) * p.nx + i;
        const T* __restrict__ Hx = p.Hn[0];   // H^{n+1/2}, just written by the H update
        const T* __restrict__ Hy = p.Hn[1];
        const T* __restrict__ Hz = p.Hn[2];
        const T* __restrict__ Ex = p.E[0];    // E^n
        const T* __restrict__ Ey = p.E[1];
        const T* __restrict__ Ez = p.E[2];
        const bool im = i > 0, jm = j > 0, km = k > 0;
        const T hx = Hx[id], hy = Hy[id], hz = Hz[id];
        const T hz_j = jm ? Hz[id - p.nx] : T(0), hy_k = km ? Hy[id - p.plane] : T(0);
        const T hx_k = km ? Hx[id - p.plane] : T(0), hz_i = im ? Hz[id - 1] : T(0);
        const T hy_i = im ? Hy[id - 1] : T(0), hx_j = jm ? Hx[id - p.nx] : T(0);
        const T ex0 = Ex[id], ey0 = Ey[id], ez0 = Ez[id];
        const long long dv = ((long long)(k - p.db[4]) * p.dny + (j - p.db[2])) * p.dnx + (i - p.db[0]);
        // each component is a design sample when its voxel is in that component's sample box and not
        // in the gap; otherwise it takes the background update
        const bool gap = in_box(p.gb, i, j, k);
        const bool dsx = !gap && in_box(p.mb[0], i, j, k), dsy = !gap && in_box(p.mb[1], i, j, k);
        const bool dsz = !gap && in_box(p.mb[2], i, j, k);
        const T idx = p.inv_dx;
        T dxv = ((hz - hz_j) - (hy - hy_k)) * idx;
        T dyv = ((hx - hx_k) - (hz - hz_i)) * idx;
        T dzv = ((hy - hy_i) - (hx - hx_j)) * idx;
        if (i == p.tfsf_i0) dzv -= __ldg(p.hinc + n) * idx;
        if (p.nb > 0 && in_box(p.sb, i, j, k)) {
            dxv += point_drive(p, i, j, k, 0, n);
            dyv += point_drive(p, i, j, k, 1, n);
            dzv += point_drive(p, i, j, k, 2, n);
        }
        T ex, ey, ez, dqx = T(0), dqy = T(0), dqz = T(0);
        ex = dsx ? design_sample<T, MP>(p, 0, p.rhoc[0][dv], dv, ex0, dxv, dqx) : p.bg_ca[0] * ex0 + p.bg_cb[0] * dxv;
        ey = dsy ? design_sample<T, MP>(p, 1, p.rhoc[1][dv], dv, ey0, dyv, dqy) : p.bg_ca[1] * ey0 + p.bg_cb[1] * dyv;
        ez = dsz ? design_sample<T, MP>(p, 2, p.rhoc[2][dv], dv, ez0, dzv, dqz) : p.bg_ca[2] * ez0 + p.bg_cb[2] * dzv;
        if (!(jm && km)) ex = ex0;
        if (!(km && im)) ey = ey0;
        if (!(im && jm)) ez = ez0;
        p.En[0][id] = ex;
        p.En[1][id] = ey;
        p.En[2][id] = ez;
        const long long slot = (long long)((n - p.snap0) % p.K) * 3 * p.nd + dv;
        T* __restrict__ snap = p.snap + slot;
        snap[0] = ex;
        snap[p.nd] = ey;
        snap[2 * p.nd] = ez;
        if (p.hist_dq) {                  // paper mode, recompute pass
            p.hist_dq[slot] = dqx;
            p.hist_dq[slot + p.nd] = dqy;
            p.hist_dq[slot + 2 * p.nd] = dqz;
        }
        if (p.td_acc && gap) {            // paper mode, forward pass: gap samples
            const long long lg = (((long long)(k - p.gb[4]) * p.gny + (j - p.gb[2])) * p.gnx + (i - p.gb[0])) * 3;
            p.td_acc[lg] += (double)ex * (double)ex;
            p.td_acc[lg + 1] += (double)ey * (double)ey;
            p.td_acc[lg + 2] += (double)ez * (double)ez;
            T* gh = p.gap_hist + (long long)n * p.nsamp + lg;
            gh[0] = ex;
            gh[1] = ey;
            gh[2] = ez;
        }
        const T mag = fabs(ex) + fabs(ey) + fabs(ez);
        if (!(mag < p.blowup)) atomicOr(p.ctl + 2, 1);
    }
    finish_step(p.ctl, p.nblocks_d, n);
}

// ---------------------------------------------------------------------------------------------
// Blocked running DFT over the design box.  After cnt steps n0..n0+cnt-1 (n0 = ctl[0] - cnt), each
// thread owns one design voxel: it reads the cnt snapshots E^{n+1} of its three samples, forms the
// block sums sum_s E^{n0+s+1} (cos, -sin)(w_f (n0+s+1) dt) in the accumulation type A, and adds
// them to the FP64 accumulators, which are read and written once per block instead of every step.
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kReduceThreads) dft_kernel(const DParams<T> d, int cnt)
{
    const long long v = (long long)blockIdx.x * kReduceThreads + threadIdx.x;
    if (v >= d.nd) return;
    const int n0 = __ldcg(d.ctl) - cnt;
    T e[kMaxSnap][3];
#pragma unroll
    for (int s = 0; s < kMaxSnap; ++s) {
        if (s < cnt) {
            const T* sp = d.snap + (long long)((n0 + s) % d.K) * 3 * d.nd + v;
            e[s][0] = sp[0];
            e[s][1] = sp[d.nd];
            e[s][2] = sp[2 * d.nd];
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
            double2 a = *acc;
            a.x += (double)re[c];
            a.y += (double)im[c];
            *acc = a;
        }
    }
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
