// Device kernels of the CCPR time-domain adjoint gradient (arXiv 2305.00234) for sm_103a.
//
// One Yee time step is three memory-bound stencil launches plus, every kMaxSnap steps, a DFT launch:
//   h_kernel:        H^{n+1/2} = H^{n-1/2} - (dt/mu0) curl E^n                   (Eq. (Maxwells)c)
//                    with CFS-CPML psi only for cells inside the edge slabs;
//   e_bg_kernel:     E^{n+1} outside the design box: background material, CPML, sources;
//   e_design_kernel: E^{n+1} inside the design box: the conductivity and the CCPR pole currents of
//                    both materials weighted by 1-rho and rho (Eqs. (Maxwells)a,b, (eps_mixed),
//                    (sigma_mixed), (Poles_mixed)), the pole recursion
//                    Q <- Q + (alpha-1) Q + beta (E^{n+1}+E^n), and an E snapshot for the DFT;
//   dft_kernel:      the running FP64 DFT over the design box, kMaxSnap steps per update;
// and the per-voxel gradient kernel (structure of Eq. (Gradient_analytic)) with a deterministic
// warp-shuffle reduction of its squared norm.
//
// Thread layout: block (32, 8) over (x, y); x is the fastest array axis, so each warp reads and
// writes 128 contiguous bytes per field (FP32).  The H and background-E kernels give each thread
// kPZ consecutive z planes and issue every load before any store, which doubles the loads in
// flight (the kernels are latency-bound otherwise) and reuses the z neighbour from registers.
// Neighbour reads at -1 (E) / +1 (H) in x and y come from L1/L2.
//
// The step index n lives in device memory (ctl[0]) so that a captured CUDA graph of K steps
// can be replayed: every kernel reads it, and the last block of e_design_kernel (of e_bg_kernel
// when there is no design box) advances it.
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
template <typename T, int MP>
__device__ __forceinline__ T design_sample(const KParams<T>& p, int c, T rho, long long dv, T e_old, T drive)
{
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
        }
    }
    return e_new;
}

template <typename T>
__device__ __forceinline__ T point_drive(const KParams<T>& p, int i, int j, int k, int c, int n)
{
    const long long lv = ((long long)(k - p.sb[4]) * (p.sb[3] - p.sb[2]) + (j - p.sb[2])) * (p.sb[1] - p.sb[0]) + (i - p.sb[0]);
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

// A block tile [bi0, bi0+kBX) x [bj0, bj0+kBY) x [k0, k0+kPZ) is interior for the H update when
// its +1 neighbours exist and no cell lies in a CPML slab or next to the TF/SF plane.
template <typename T>
__device__ __forceinline__ bool h_block_interior(const KParams<T>& p, int bi0, int bj0, int k0)
{
    return bi0 >= p.cpl[0] && bi0 + kBX < p.nx - p.cph[0] && bj0 >= p.cpl[1] && bj0 + kBY < p.ny - p.cph[1] &&
           k0 >= p.cpl[2] && k0 + kPZ < p.nz - p.cph[2] && !(p.tfsf_i0 - 1 >= bi0 && p.tfsf_i0 - 1 < bi0 + kBX);
}

// ... and interior for the background E update when its -1 neighbours exist (no PEC wall), no cell
// lies in a CPML slab, on the TF/SF plane, in the point-source box or in the design box.
template <typename T>
__device__ __forceinline__ bool e_block_interior(const KParams<T>& p, int bi0, int bj0, int k0)
{
    const bool slab_free = bi0 >= p.cpl[0] && bi0 >= 1 && bi0 + kBX <= p.nx - p.cph[0] && bj0 >= p.cpl[1] && bj0 >= 1 &&
                           bj0 + kBY <= p.ny - p.cph[1] && k0 >= p.cpl[2] && k0 >= 1 && k0 + kPZ <= p.nz - p.cph[2];
    const bool no_plane = !(p.tfsf_i0 >= bi0 && p.tfsf_i0 < bi0 + kBX);
    const bool no_src = p.nb == 0 || p.sb[1] <= bi0 || p.sb[0] >= bi0 + kBX || p.sb[3] <= bj0 || p.sb[2] >= bj0 + kBY ||
                        p.sb[5] <= k0 || p.sb[4] >= k0 + kPZ;
    const bool no_design = p.db[1] <= bi0 || p.db[0] >= bi0 + kBX || p.db[3] <= bj0 || p.db[2] >= bj0 + kBY ||
                           p.db[5] <= k0 || p.db[4] >= k0 + kPZ;
    return slab_free && no_plane && no_src && no_design;
}

// H update, kPZ consecutive z planes per thread: all loads of both planes are issued before any
// store, and the z+1 neighbour of plane r is plane r+1's own E value.
template <typename T>
__global__ void __launch_bounds__(kBX * kBY, FDTD_H_MINB) h_kernel(const KParams<T> p)
{
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    const int k0 = blockIdx.z * kPZ;
    if (i >= p.nx || j >= p.ny) return;
    const T* __restrict__ Ex = p.E[0];
    const T* __restrict__ Ey = p.E[1];
    const T* __restrict__ Ez = p.E[2];
    T* __restrict__ Hx = p.H[0];
    T* __restrict__ Hy = p.H[1];
    T* __restrict__ Hz = p.H[2];
    if (h_block_interior(p, blockIdx.x * kBX, blockIdx.y * kBY, k0)) {
        // no wall, CPML slab or TF/SF plane anywhere in this block: plain stencil, 32-bit indices
        const int nx = p.nx, pl = (int)p.plane;
        const int id0 = (k0 * p.ny + j) * nx + i;
        T fex[kPZ + 1], fey[kPZ + 1], fez[kPZ], fexj[kPZ], fezj[kPZ], feyi[kPZ], fezi[kPZ], fhx[kPZ], fhy[kPZ], fhz[kPZ];
#pragma unroll
        for (int r = 0; r <= kPZ; ++r) {
            const int id = id0 + r * pl;
            fex[r] = Ex[id];
            fey[r] = Ey[id];
            if (r < kPZ) {
                fez[r] = Ez[id];
                fexj[r] = Ex[id + nx];
                fezj[r] = Ez[id + nx];
                feyi[r] = Ey[id + 1];
                fezi[r] = Ez[id + 1];
                fhx[r] = Hx[id];
                fhy[r] = Hy[id];
                fhz[r] = Hz[id];
            }
        }
        const T c = p.ch * p.inv_dx;
#pragma unroll
        for (int r = 0; r < kPZ; ++r) {
            const int id = id0 + r * pl;
            Hx[id] = fhx[r] - c * ((fezj[r] - fez[r]) - (fey[r + 1] - fey[r]));
            Hy[id] = fhy[r] - c * ((fex[r + 1] - fex[r]) - (fezi[r] - fez[r]));
            Hz[id] = fhz[r] - c * ((feyi[r] - fey[r]) - (fexj[r] - fex[r]));
        }
        return;
    }
    const bool ip = i + 1 < p.nx, jp = j + 1 < p.ny;
    T ex[kPZ + 1], ey[kPZ + 1];
    T ez[kPZ], ex_j[kPZ], ez_j[kPZ], ey_i[kPZ], ez_i[kPZ], hx[kPZ], hy[kPZ], hz[kPZ];
#pragma unroll
    for (int r = 0; r <= kPZ; ++r) {
        const int k = k0 + r;
        const bool ok = k < p.nz;
        const long long id = ((long long)k * p.ny + j) * p.nx + i;
        ex[r] = ok ? Ex[id] : T(0);     // beyond the last plane: PEC wall
        ey[r] = ok ? Ey[id] : T(0);
        if (r < kPZ) {
            ez[r] = ok ? Ez[id] : T(0);
            ex_j[r] = ok && jp ? Ex[id + p.nx] : T(0);
            ez_j[r] = ok && jp ? Ez[id + p.nx] : T(0);
            ey_i[r] = ok && ip ? Ey[id + 1] : T(0);
            ez_i[r] = ok && ip ? Ez[id + 1] : T(0);
            hx[r] = ok ? Hx[id] : T(0);
            hy[r] = ok ? Hy[id] : T(0);
            hz[r] = ok ? Hz[id] : T(0);
        }
    }
    const int sx = slab_index(i, p.cpl[0], p.cph[0], p.nx);
    const int sy = slab_index(j, p.cpl[1], p.cph[1], p.ny);
    const T idx = p.inv_dx, ch = p.ch;
#pragma unroll
    for (int r = 0; r < kPZ; ++r) {
        const int k = k0 + r;
        if (k >= p.nz) break;
        const long long id = ((long long)k * p.ny + j) * p.nx + i;
        const int sz = slab_index(k, p.cpl[2], p.cph[2], p.nz);
        // H_x at (i, j+1/2, k+1/2): (curl E)_x = dEz/dy - dEy/dz
        T xa = (ez_j[r] - ez[r]) * idx, xb = (ey[r + 1] - ey[r]) * idx;
        // H_y at (i+1/2, j, k+1/2): (curl E)_y = dEx/dz - dEz/dx
        T ya = (ex[r + 1] - ex[r]) * idx, yb = (ez_i[r] - ez[r]) * idx;
        // H_z at (i+1/2, j+1/2, k): (curl E)_z = dEy/dx - dEx/dy
        T za = (ey_i[r] - ey[r]) * idx, zb = (ex_j[r] - ex[r]) * idx;
        if (i == p.tfsf_i0 - 1) yb -= __ldg(p.einc + read_step<T>(p.ctl)) * idx;   // H_y here is scattered field
        if (sy >= 0) {
            xa = stretch(xa, p.pmlH[1], sy, p.psiH[0][0] + psi_index(p, i, j, k, 1, sy));
            zb = stretch(zb, p.pmlH[1], sy, p.psiH[2][1] + psi_index(p, i, j, k, 1, sy));
        }
        if (sz >= 0) {
            xb = stretch(xb, p.pmlH[2], sz, p.psiH[0][1] + psi_index(p, i, j, k, 2, sz));
            ya = stretch(ya, p.pmlH[2], sz, p.psiH[1][0] + psi_index(p, i, j, k, 2, sz));
        }
        if (sx >= 0) {
            yb = stretch(yb, p.pmlH[0], sx, p.psiH[1][1] + psi_index(p, i, j, k, 0, sx));
            za = stretch(za, p.pmlH[0], sx, p.psiH[2][0] + psi_index(p, i, j, k, 0, sx));
        }
        Hx[id] = hx[r] - ch * (xa - xb);
        Hy[id] = hy[r] - ch * (ya - yb);
        Hz[id] = hz[r] - ch * (za - zb);
    }
}

// E update outside the design box (background material, CPML slabs, sources), kPZ planes per
// thread.  Cells inside the design box are left to e_design_kernel; blocks wholly inside it exit.
template <typename T>
__global__ void __launch_bounds__(kBX * kBY, FDTD_EBG_MINB) e_bg_kernel(const KParams<T> p)
{
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    const int k0 = blockIdx.z * kPZ;
    const int n = read_step<T>(p.ctl);
    const int bi0 = blockIdx.x * kBX, bj0 = blockIdx.y * kBY;
    const bool block_in_design = bi0 >= p.db[0] && bi0 + kBX <= p.db[1] && bj0 >= p.db[2] && bj0 + kBY <= p.db[3] &&
                                 k0 >= p.db[4] && k0 + kPZ <= p.db[5];
    if (!block_in_design && e_block_interior(p, bi0, bj0, k0)) {
        if (i < p.nx && j < p.ny) {   // plain stencil, 32-bit indices
            const T* __restrict__ Hx = p.H[0];
            const T* __restrict__ Hy = p.H[1];
            const T* __restrict__ Hz = p.H[2];
            T* __restrict__ Ex = p.E[0];
            T* __restrict__ Ey = p.E[1];
            T* __restrict__ Ez = p.E[2];
            const int nx = p.nx, pl = (int)p.plane;
            const int id0 = (k0 * p.ny + j) * nx + i;
            T fhx[kPZ + 1], fhy[kPZ + 1], fhz[kPZ], fhzj[kPZ], fhzi[kPZ], fhyi[kPZ], fhxj[kPZ], fe[kPZ][3];
#pragma unroll
            for (int r = 0; r <= kPZ; ++r) {
                const int id = id0 + (r - 1) * pl;
                fhx[r] = Hx[id];
                fhy[r] = Hy[id];
                if (r > 0) {
                    const int q = r - 1;
                    fhz[q] = Hz[id];
                    fhzj[q] = Hz[id - nx];
                    fhxj[q] = Hx[id - nx];
                    fhzi[q] = Hz[id - 1];
                    fhyi[q] = Hy[id - 1];
                    fe[q][0] = Ex[id];
                    fe[q][1] = Ey[id];
                    fe[q][2] = Ez[id];
                }
            }
            const T idx = p.inv_dx;
            T emax = T(0);
#pragma unroll
            for (int r = 0; r < kPZ; ++r) {
                const int id = id0 + r * pl;
                const T ex = p.bg_ca[0] * fe[r][0] + p.bg_cb[0] * idx * ((fhz[r] - fhzj[r]) - (fhy[r + 1] - fhy[r]));
                const T ey = p.bg_ca[1] * fe[r][1] + p.bg_cb[1] * idx * ((fhx[r + 1] - fhx[r]) - (fhz[r] - fhzi[r]));
                const T ez = p.bg_ca[2] * fe[r][2] + p.bg_cb[2] * idx * ((fhy[r + 1] - fhyi[r]) - (fhx[r + 1] - fhxj[r]));
                Ex[id] = ex;
                Ey[id] = ey;
                Ez[id] = ez;
                emax = fmax(emax, fabs(ex) + fabs(ey) + fabs(ez));
            }
            if (!(emax < p.blowup)) atomicOr(p.ctl + 2, 1);
        }
    } else if (!block_in_design && i < p.nx && j < p.ny) {
        const T* __restrict__ Hx = p.H[0];
        const T* __restrict__ Hy = p.H[1];
        const T* __restrict__ Hz = p.H[2];
        T* __restrict__ Ex = p.E[0];
        T* __restrict__ Ey = p.E[1];
        T* __restrict__ Ez = p.E[2];
        const bool im = i > 0, jm = j > 0;
        T hx[kPZ + 1], hy[kPZ + 1];     // index 0 = plane k0-1 (the z-1 neighbour of the first plane)
        T hz[kPZ], hz_j[kPZ], hz_i[kPZ], hy_i[kPZ], hx_j[kPZ], e0[kPZ][3];
#pragma unroll
        for (int r = 0; r <= kPZ; ++r) {
            const int k = k0 + r - 1;
            const bool ok = k >= 0 && k < p.nz;
            const long long id = ((long long)k * p.ny + j) * p.nx + i;
            hx[r] = ok ? Hx[id] : T(0);
            hy[r] = ok ? Hy[id] : T(0);
            if (r > 0) {
                const int q = r - 1;
                hz[q] = ok ? Hz[id] : T(0);
                hz_j[q] = ok && jm ? Hz[id - p.nx] : T(0);
                hx_j[q] = ok && jm ? Hx[id - p.nx] : T(0);
                hz_i[q] = ok && im ? Hz[id - 1] : T(0);
                hy_i[q] = ok && im ? Hy[id - 1] : T(0);
                e0[q][0] = ok ? Ex[id] : T(0);
                e0[q][1] = ok ? Ey[id] : T(0);
                e0[q][2] = ok ? Ez[id] : T(0);
            }
        }
        const int sx = slab_index(i, p.cpl[0], p.cph[0], p.nx);
        const int sy = slab_index(j, p.cpl[1], p.cph[1], p.ny);
        const T idx = p.inv_dx;
        T emax = T(0);
#pragma unroll
        for (int r = 0; r < kPZ; ++r) {
            const int k = k0 + r;
            if (k >= p.nz || in_box(p.db, i, j, k)) continue;
            const long long id = ((long long)k * p.ny + j) * p.nx + i;
            const bool km = k > 0;
            const int sz = slab_index(k, p.cpl[2], p.cph[2], p.nz);
            // E_x: dHz/dy - dHy/dz ; E_y: dHx/dz - dHz/dx ; E_z: dHy/dx - dHx/dy
            T xa = (hz[r] - hz_j[r]) * idx, xb = (hy[r + 1] - hy[r]) * idx;
            T ya = (hx[r + 1] - hx[r]) * idx, yb = (hz[r] - hz_i[r]) * idx;
            T za = (hy[r + 1] - hy_i[r]) * idx, zb = (hx[r + 1] - hx_j[r]) * idx;
            if (i == p.tfsf_i0) za -= __ldg(p.hinc + n) * idx;    // H_y(i0-1/2) is scattered field
            if (sy >= 0) {
                xa = stretch(xa, p.pmlE[1], sy, p.psiE[0][0] + psi_index(p, i, j, k, 1, sy));
                zb = stretch(zb, p.pmlE[1], sy, p.psiE[2][1] + psi_index(p, i, j, k, 1, sy));
            }
            if (sz >= 0) {
                xb = stretch(xb, p.pmlE[2], sz, p.psiE[0][1] + psi_index(p, i, j, k, 2, sz));
                ya = stretch(ya, p.pmlE[2], sz, p.psiE[1][0] + psi_index(p, i, j, k, 2, sz));
            }
            if (sx >= 0) {
                yb = stretch(yb, p.pmlE[0], sx, p.psiE[1][1] + psi_index(p, i, j, k, 0, sx));
                za = stretch(za, p.pmlE[0], sx, p.psiE[2][0] + psi_index(p, i, j, k, 0, sx));
            }
            T dxv = xa - xb, dyv = ya - yb, dzv = za - zb;
            if (p.nb > 0 && in_box(p.sb, i, j, k)) {
                dxv += point_drive(p, i, j, k, 0, n);
                dyv += point_drive(p, i, j, k, 1, n);
                dzv += point_drive(p, i, j, k, 2, n);
            }
            T ex = p.bg_ca[0] * e0[r][0] + p.bg_cb[0] * dxv;
            T ey = p.bg_ca[1] * e0[r][1] + p.bg_cb[1] * dyv;
            T ez = p.bg_ca[2] * e0[r][2] + p.bg_cb[2] * dzv;
            // PEC walls: components tangential to a wall at index 0 stay zero
            if (!(jm && km)) ex = e0[r][0];
            if (!(km && im)) ey = e0[r][1];
            if (!(im && jm)) ez = e0[r][2];
            Ex[id] = ex;
            Ey[id] = ey;
            Ez[id] = ez;
            emax = fmax(emax, fabs(ex) + fabs(ey) + fabs(ez));
        }
        if (!(emax < p.blowup)) atomicOr(p.ctl + 2, 1);
    }
    if (p.nd == 0) finish_step(p.ctl, p.nblocks_e, n);
}

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
        const T* __restrict__ Hx = p.H[0];
        const T* __restrict__ Hy = p.H[1];
        const T* __restrict__ Hz = p.H[2];
        T* __restrict__ Ex = p.E[0];
        T* __restrict__ Ey = p.E[1];
        T* __restrict__ Ez = p.E[2];
        const bool im = i > 0, jm = j > 0, km = k > 0;
        const T hx = Hx[id], hy = Hy[id], hz = Hz[id];
        const T hz_j = jm ? Hz[id - p.nx] : T(0), hy_k = km ? Hy[id - p.plane] : T(0);
        const T hx_k = km ? Hx[id - p.plane] : T(0), hz_i = im ? Hz[id - 1] : T(0);
        const T hy_i = im ? Hy[id - 1] : T(0), hx_j = jm ? Hx[id - p.nx] : T(0);
        const T ex0 = Ex[id], ey0 = Ey[id], ez0 = Ez[id];
        const long long dv = ((long long)(k - p.db[4]) * p.dny + (j - p.db[2])) * p.dnx + (i - p.db[0]);
        const bool design = !in_box(p.gb, i, j, k);
        const T rho = design ? p.rho[dv] : T(0);
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
        T ex, ey, ez;
        if (design) {
            ex = design_sample<T, MP>(p, 0, rho, dv, ex0, dxv);
            ey = design_sample<T, MP>(p, 1, rho, dv, ey0, dyv);
            ez = design_sample<T, MP>(p, 2, rho, dv, ez0, dzv);
        } else {
            ex = p.bg_ca[0] * ex0 + p.bg_cb[0] * dxv;
            ey = p.bg_ca[1] * ey0 + p.bg_cb[1] * dyv;
            ez = p.bg_ca[2] * ez0 + p.bg_cb[2] * dzv;
        }
        if (!(jm && km)) ex = ex0;
        if (!(km && im)) ey = ey0;
        if (!(im && jm)) ez = ez0;
        Ex[id] = ex;
        Ey[id] = ey;
        Ez[id] = ez;
        T* __restrict__ snap = p.snap + (long long)(n % p.K) * 3 * p.nd + dv;
        snap[0] = ex;
        snap[p.nd] = ey;
        snap[2 * p.nd] = ez;
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
    const long long v = (long long)blockIdx.x * kReduceThreads + threadIdx.x;
    double G = 0.0;
    if (v < g.nd) {
        const int i = g.db[0] + (int)(v % g.dnx);
        const int j = g.db[2] + (int)((v / g.dnx) % g.dny);
        const int k = g.db[4] + (int)(v / ((long long)g.dnx * g.dny));
        if (!in_box(g.gb, i, j, k)) {
            const double s = 1.0 - 2.0 * (double)g.rho[v];
            for (int c = 0; c < 3; ++c)
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
        if (g.grad64) g.grad64[v] = G;
        if (g.grad32) g.grad32[v] = (float)G;
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

}  // namespace fdtd
