// Shell kernels on x-adjacent cell pairs (FP32).  The same cell updates as h_column / e_column in
// fdtd_step.cuh (Eqs. (Maxwells)a-c with the background material, CFS-CPML psi in the edge slabs, the
// TF/SF correction, point sources, PEC walls), with each thread updating the two cells (x, x+1) of a pair:
// 8-byte loads and stores, and Blackwell's paired FP32 instructions (one instruction for both cells).
// The H update is per element the scalar one, operation for operation and explicitly rounded, so an H
// value is the same whichever kernel stores it (the fused interior kernel recomputes its -x/-y halo H and
// relies on that).  The E update takes the same explicitly rounded form as the fused interior kernel.
//
// Used when every pair lies on one side of each x boundary of the CPML and of the shell boxes: nx, the x CPML
// thicknesses and the shell boxes' x bounds all even (the host checks; otherwise the scalar shell kernels
// run).  A pair may straddle the working box's x bounds (the E kernel then stores only its outside cell),
// the TF/SF plane and a point source.
#pragma once
#include "fdtd_step.cuh"

#ifndef FDTD_SHELL2_PZ
#define FDTD_SHELL2_PZ 1
#endif
#ifndef FDTD_SHELL2_MINB
#define FDTD_SHELL2_MINB 4
#endif

namespace fdtd {

constexpr int kShell2PZ = FDTD_SHELL2_PZ;   // z planes per batch of loads (pairs hold twice a column's values)
static_assert(kShellKZ % kShell2PZ == 0, "column depth a multiple of the batch");

__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }

// L2 prefetch of the field rows a column needs FDTD_SHELL2_PF_H / _E planes ahead in the H / E kernel (0:
// none): the loads of the coming planes then find their lines in L2 instead of waiting on HBM, without
// holding registers.
#ifndef FDTD_SHELL2_PF_H
#define FDTD_SHELL2_PF_H 0
#endif
#ifndef FDTD_SHELL2_PF_E
#define FDTD_SHELL2_PF_E 1   // measured: E kernel 0.0616 -> 0.0610 ms on the config-2 grid; the H kernel slows
#endif
__device__ __forceinline__ void pf_l2(const float* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 ldp(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void stp(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }

// The pair (x, x+1), x = B[0] + 2j, of block b / thread t of a paired shell launch (boxes counted in pairs).
__device__ __forceinline__ bool shell_pair(const ShellBoxes& s, ShellCol& c)
{
    int q = 0;
    while (q + 1 < s.n && blockIdx.x >= s.first[q + 1]) ++q;
    const int* B = s.b[q];
    const unsigned loc = blockIdx.x - s.first[q];
    const unsigned wx = (unsigned)(B[1] - B[0]) / 2u, wxy = wx * (B[3] - B[2]);
    const unsigned chunks = (wxy + kShellCells - 1) / kShellCells;
    const unsigned zc = loc / chunks;
    const unsigned t = (loc - zc * chunks) * kShellCells + threadIdx.y * kBX + threadIdx.x;
    const unsigned yy = t / wx;
    c.x = B[0] + 2 * (int)(t - yy * wx);
    c.y = B[2] + (int)yy;
    c.k0 = B[4] + (int)zc * s.kz;
    c.k1 = min(B[5], c.k0 + s.kz);
    return t < wxy;
}

// {1/kappa, b, c}: per element of slab indices s, s + 1 (x slab), or the same for both (y, z slabs).
__device__ __forceinline__ void pml_pair(const float* __restrict__ tab, int s, int ds, float2& kinv, float2& b, float2& c)
{
    const float4 u = __ldg(reinterpret_cast<const float4*>(tab) + s);
    const float4 v = ds ? __ldg(reinterpret_cast<const float4*>(tab) + s + 1) : u;
    kinv = f2(u.x, v.x);
    b = f2(u.y, v.y);
    c = f2(u.z, v.z);
}

// d -> d/kappa + psi', psi' = b psi + c d, per element as stretch_v.
__device__ __forceinline__ float2 stretch_p(float2 d, const float* __restrict__ tab, int s, int ds, float2& psi)
{
    float2 kinv, b, c;
    pml_pair(tab, s, ds, kinv, b, c);
    psi = p_add(p_mul(b, psi), p_mul(c, d));
    return p_add(p_mul(d, kinv), psi);
}

__device__ __forceinline__ void psi_load_p(float* const (&ps)[3][2], const PsiCol& pc, unsigned k, unsigned plane,
                                           unsigned col, int sx, int sy, int sz, float2 (&v)[6])
{
    const unsigned q1 = k * pc.qys + pc.qy0, q2 = (unsigned)max(sz, 0) * plane + col, q0 = k * pc.qxs + pc.qx0;
    const float2 z = f2(0.f, 0.f);
    v[0] = sy >= 0 ? ldp(ps[0][0] + q1) : z;
    v[1] = sy >= 0 ? ldp(ps[2][1] + q1) : z;
    v[2] = sz >= 0 ? ldp(ps[0][1] + q2) : z;
    v[3] = sz >= 0 ? ldp(ps[1][0] + q2) : z;
    v[4] = sx >= 0 ? ldp(ps[1][1] + q0) : z;
    v[5] = sx >= 0 ? ldp(ps[2][0] + q0) : z;
}

__device__ __forceinline__ void psi_store_p(float* const (&ps)[3][2], const PsiCol& pc, unsigned k, unsigned plane,
                                            unsigned col, int sx, int sy, int sz, const float2 (&v)[6])
{
    if (sy >= 0) {
        const unsigned q = k * pc.qys + pc.qy0;
        stp(ps[0][0] + q, v[0]);
        stp(ps[2][1] + q, v[1]);
    }
    if (sz >= 0) {
        const unsigned q = (unsigned)sz * plane + col;
        stp(ps[0][1] + q, v[2]);
        stp(ps[1][0] + q, v[3]);
    }
    if (sx >= 0) {
        const unsigned q = k * pc.qxs + pc.qx0;
        stp(ps[1][1] + q, v[4]);
        stp(ps[2][0] + q, v[5]);
    }
}

// H of the shell, one pair of columns per thread, planes [k0, k1) in batches of kShell2PZ.
__global__ void __launch_bounds__(kBX * kBY, FDTD_SHELL2_MINB) shell_h2_kernel(const KParams<float> p, const ShellBoxes s)
{
    constexpr int P = kShell2PZ;
    pdl_wait();
    pdl_trigger();
    ShellCol cl;
    if (!shell_pair(s, cl)) return;
    const int x = cl.x, y = cl.y;
    const int n = read_step<float>(p.ctl);
    const float cneg = -(p.ch * p.inv_dx), idx = p.inv_dx, ch = p.ch;
    const float2 cn = f2(cneg, cneg), idx2 = f2(idx, idx), ch2 = f2(ch, ch);
    const float einc_n = p.tfsf_i0 >= 0 ? __ldg(p.einc + n) : 0.f;
    // TF/SF: H_y left of the plane is scattered field; the other element subtracts +0 (exact)
    const float2 einc2 = f2(x == p.tfsf_i0 - 1 ? einc_n : 0.f, x + 1 == p.tfsf_i0 - 1 ? einc_n : 0.f);
    const bool tf = x == p.tfsf_i0 - 1 || x + 1 == p.tfsf_i0 - 1;
    const float2 einc2i = f2(x == p.tfsf_i0 - 1 ? __fmul_rn(einc_n, idx) : 0.f,
                             x + 1 == p.tfsf_i0 - 1 ? __fmul_rn(einc_n, idx) : 0.f);
    const int sx = slab_index(x, p.cpl[0], p.cph[0], p.nx), sy = slab_index(y, p.cpl[1], p.cph[1], p.ny);
    const bool xp = x + 2 < p.nx, yp = y + 1 < p.ny;
    const unsigned nx = (unsigned)p.nx, plane = (unsigned)p.plane, col = (unsigned)y * nx + (unsigned)x;
    const PsiCol pc = psi_col(p, x, y, sx, sy);
    const float* __restrict__ E0 = p.E[0];
    const float* __restrict__ E1 = p.E[1];
    const float* __restrict__ E2 = p.E[2];
    const float2 z2 = f2(0.f, 0.f);
    float2 exc = ldp(E0 + (unsigned)cl.k0 * plane + col), eyc = ldp(E1 + (unsigned)cl.k0 * plane + col);
    for (int it = 0; it < kShellKZ / P; ++it) {
        const int kb = cl.k0 + it * P;
        if (kb >= cl.k1) break;
        float2 ex0[P], ey0[P], ez0[P], ezy[P], exy[P], ezx[P], eyx[P], exz[P], eyz[P], ho[P][3], ps[P][6];
        int sz[P];
#pragma unroll
        for (int r = 0; r < P; ++r) {
            const int k = kb + r;
            sz[r] = slab_index(k, p.cpl[2], p.cph[2], p.nz);
            if (k >= cl.k1) continue;
            const unsigned id = (unsigned)k * plane + col;
            const bool zp = k + 1 < p.nz;
            if (FDTD_SHELL2_PF_H > 0 && k + FDTD_SHELL2_PF_H < cl.k1) {
                const unsigned ip = id + FDTD_SHELL2_PF_H * plane;
                pf_l2(p.H[0] + ip);
                pf_l2(p.H[1] + ip);
                pf_l2(p.H[2] + ip);
                if (k + FDTD_SHELL2_PF_H + 1 < p.nz) {
                    pf_l2(E0 + ip + plane);
                    pf_l2(E1 + ip + plane);
                    pf_l2(E2 + ip + plane);
                }
            }
            ex0[r] = r == 0 ? exc : exz[r - 1];
            ey0[r] = r == 0 ? eyc : eyz[r - 1];
            ez0[r] = ldp(E2 + id);
            const float ezn = xp ? E2[id + 2] : 0.f, eyn = xp ? E1[id + 2] : 0.f;
            ezx[r] = f2(ez0[r].y, ezn);
            eyx[r] = f2(ey0[r].y, eyn);
            ezy[r] = yp ? ldp(E2 + id + nx) : z2;
            exy[r] = yp ? ldp(E0 + id + nx) : z2;
            exz[r] = zp ? ldp(E0 + id + plane) : z2;
            eyz[r] = zp ? ldp(E1 + id + plane) : z2;
            ho[r][0] = ldp(p.H[0] + id);
            ho[r][1] = ldp(p.H[1] + id);
            ho[r][2] = ldp(p.H[2] + id);
            psi_load_p(p.psiH, pc, (unsigned)k, plane, col, sx, sy, sz[r], ps[r]);
        }
#pragma unroll
        for (int r = 0; r < P; ++r) {
            const int k = kb + r;
            if (k >= cl.k1) continue;
            const unsigned id = (unsigned)k * plane + col;
            float2 hx, hy, hz;
            if (sx < 0 && sy < 0 && sz[r] < 0) {   // h_cheap per element
                float2 dyx = p_sub(ezx[r], ez0[r]);
                if (tf) dyx = p_sub(dyx, einc2);
                hx = p_fma(cn, p_sub(p_sub(ezy[r], ez0[r]), p_sub(eyz[r], ey0[r])), ho[r][0]);
                hy = p_fma(cn, p_sub(p_sub(exz[r], ex0[r]), dyx), ho[r][1]);
                hz = p_fma(cn, p_sub(p_sub(eyx[r], ey0[r]), p_sub(exy[r], ex0[r])), ho[r][2]);
            } else {
                float2 xa = p_mul(p_sub(ezy[r], ez0[r]), idx2), xb = p_mul(p_sub(eyz[r], ey0[r]), idx2);
                float2 ya = p_mul(p_sub(exz[r], ex0[r]), idx2), yb = p_mul(p_sub(ezx[r], ez0[r]), idx2);
                float2 za = p_mul(p_sub(eyx[r], ey0[r]), idx2), zb = p_mul(p_sub(exy[r], ex0[r]), idx2);
                if (tf) yb = p_sub(yb, einc2i);
                if (sy >= 0) {
                    xa = stretch_p(xa, p.pmlH[1], sy, 0, ps[r][0]);
                    zb = stretch_p(zb, p.pmlH[1], sy, 0, ps[r][1]);
                }
                if (sz[r] >= 0) {
                    xb = stretch_p(xb, p.pmlH[2], sz[r], 0, ps[r][2]);
                    ya = stretch_p(ya, p.pmlH[2], sz[r], 0, ps[r][3]);
                }
                if (sx >= 0) {
                    yb = stretch_p(yb, p.pmlH[0], sx, 1, ps[r][4]);
                    za = stretch_p(za, p.pmlH[0], sx, 1, ps[r][5]);
                }
                hx = p_sub(ho[r][0], p_mul(ch2, p_sub(xa, xb)));
                hy = p_sub(ho[r][1], p_mul(ch2, p_sub(ya, yb)));
                hz = p_sub(ho[r][2], p_mul(ch2, p_sub(za, zb)));
                psi_store_p(p.psiHn, pc, (unsigned)k, plane, col, sx, sy, sz[r], ps[r]);
            }
            stp(p.Hn[0] + id, hx);
            stp(p.Hn[1] + id, hy);
            stp(p.Hn[2] + id, hz);
        }
        exc = exz[P - 1];   // read only when plane kb + P is this thread's
        eyc = eyz[P - 1];
    }
}

// E of the shell cells outside the working box, one pair of columns per thread.  It may run concurrently
// with the design-E kernel: the last block of the two launches advances the step.
__global__ void __launch_bounds__(kBX * kBY, FDTD_SHELL2_MINB) shell_e2_kernel(const KParams<float> p, const ShellBoxes s)
{
    constexpr int P = kShell2PZ;
    pdl_wait();
    pdl_trigger();
    ShellCol cl;
    const bool live = shell_pair(s, cl);
    const int n = read_step<float>(p.ctl);
    if (live) {
        const int x = cl.x, y = cl.y;
        const float hinc_n = p.tfsf_i0 >= 0 ? __ldg(p.hinc + n) : 0.f;
        const bool check = (n & 15) == 0 || n + 1 == p.n_steps;
        const bool tf0 = x == p.tfsf_i0, tf1 = x + 1 == p.tfsf_i0;   // H_y(i0-1/2) is scattered field
        const bool tf = tf0 || tf1;
        const int sx = slab_index(x, p.cpl[0], p.cph[0], p.nx), sy = slab_index(y, p.cpl[1], p.cph[1], p.ny);
        const unsigned nx = (unsigned)p.nx, plane = (unsigned)p.plane, col = (unsigned)y * nx + (unsigned)x;
        const PsiCol pc = psi_col(p, x, y, sx, sy);
        // cells of the working box are the design-E kernel's; a pair may straddle its x bounds
        const bool in_y = y >= p.db[2] && y < p.db[3];
        const bool in_dx0 = in_y && x >= p.db[0] && x < p.db[1], in_dx1 = in_y && x + 1 >= p.db[0] && x + 1 < p.db[1];
        const float idx = p.inv_dx;
        const float2 idx2 = f2(idx, idx), z2 = f2(0.f, 0.f);
        const float2 hinc2 = f2(tf0 ? hinc_n : 0.f, tf1 ? hinc_n : 0.f);
        const float2 hinc2i = f2(tf0 ? __fmul_rn(hinc_n, idx) : 0.f, tf1 ? __fmul_rn(hinc_n, idx) : 0.f);
        float2 ca[3], cbi[3], cb[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ca[c] = f2(p.bg_ca[c], p.bg_ca[c]);
            cbi[c] = f2(p.bg_cbi[c], p.bg_cbi[c]);
            cb[c] = f2(p.bg_cb[c], p.bg_cb[c]);
        }
        const float* __restrict__ H0 = p.Hn[0];
        const float* __restrict__ H1 = p.Hn[1];
        const float* __restrict__ H2 = p.Hn[2];
        float2 hxb = z2, hyb = z2;   // H_x, H_y of the plane below the batch
        if (cl.k0 > 0) {
            hxb = ldp(H0 + (unsigned)(cl.k0 - 1) * plane + col);
            hyb = ldp(H1 + (unsigned)(cl.k0 - 1) * plane + col);
        }
        float emax = 0.f;
        for (int kb = cl.k0; kb < cl.k1; kb += P) {
            float2 h[P][3], hzy[P], hxy[P], hzx[P], hyx[P], e0[P][3], ps[P][6];
            bool on0[P], on1[P];
            int sz[P];
#pragma unroll
            for (int r = 0; r < P; ++r) {
                const int k = kb + r;
                sz[r] = slab_index(k, p.cpl[2], p.cph[2], p.nz);
                const bool in_dz = k >= p.db[4] && k < p.db[5];
                on0[r] = k < cl.k1 && !(in_dx0 && in_dz);
                on1[r] = k < cl.k1 && !(in_dx1 && in_dz);
                if (k >= cl.k1) continue;
                const unsigned id = (unsigned)k * plane + col;
                if (FDTD_SHELL2_PF_E > 0 && k + FDTD_SHELL2_PF_E < cl.k1) {
                    const unsigned ip = id + FDTD_SHELL2_PF_E * plane;
                    pf_l2(H0 + ip);
                    pf_l2(H1 + ip);
                    pf_l2(H2 + ip);
                    pf_l2(p.E[0] + ip);
                    pf_l2(p.E[1] + ip);
                    pf_l2(p.E[2] + ip);
                }
                h[r][0] = ldp(H0 + id);
                h[r][1] = ldp(H1 + id);
                h[r][2] = ldp(H2 + id);
                hzy[r] = y > 0 ? ldp(H2 + id - nx) : z2;                  // H_z(y-1)
                hxy[r] = y > 0 ? ldp(H0 + id - nx) : z2;                  // H_x(y-1)
                hzx[r] = f2(x > 0 ? H2[id - 1] : 0.f, h[r][2].x);        // H_z(x-1)
                hyx[r] = f2(x > 0 ? H1[id - 1] : 0.f, h[r][1].x);        // H_y(x-1)
                e0[r][0] = ldp(p.E[0] + id);
                e0[r][1] = ldp(p.E[1] + id);
                e0[r][2] = ldp(p.E[2] + id);
                psi_load_p(p.psiE, pc, (unsigned)k, plane, col, sx, sy, sz[r], ps[r]);
            }
#pragma unroll
            for (int r = 0; r < P; ++r) {
                const int k = kb + r;
                const float2 hxz = r == 0 ? hxb : h[r - 1][0], hyz = r == 0 ? hyb : h[r - 1][1];
                if (!on0[r] && !on1[r]) continue;
                const unsigned id = (unsigned)k * plane + col;
                const float2 rxa = p_sub(h[r][2], hzy[r]), rxb = p_sub(h[r][1], hyz);
                const float2 rya = p_sub(h[r][0], hxz), ryb = p_sub(h[r][2], hzx[r]);
                const float2 rza = p_sub(h[r][1], hyx[r]), rzb = p_sub(h[r][0], hxy[r]);
                const bool src0 = p.nb > 0 && in_box(p.sb, x, y, k), src1 = p.nb > 0 && in_box(p.sb, x + 1, y, k);
                float2 ex, ey, ez;
                if (sx < 0 && sy < 0 && sz[r] < 0 && !src0 && !src1 && x > 0 && y > 0 && k > 0) {
                    ex = p_fma(ca[0], e0[r][0], p_mul(cbi[0], p_sub(rxa, rxb)));
                    ey = p_fma(ca[1], e0[r][1], p_mul(cbi[1], p_sub(rya, ryb)));
                    ez = p_fma(ca[2], e0[r][2], p_mul(cbi[2], p_sub(tf ? p_sub(rza, hinc2) : rza, rzb)));
                } else {
                    float2 xa = p_mul(rxa, idx2), xb = p_mul(rxb, idx2), ya = p_mul(rya, idx2), yb = p_mul(ryb, idx2);
                    float2 za = p_mul(rza, idx2), zb = p_mul(rzb, idx2);
                    if (tf) za = p_sub(za, hinc2i);
                    if (sy >= 0) {
                        xa = stretch_p(xa, p.pmlE[1], sy, 0, ps[r][0]);
                        zb = stretch_p(zb, p.pmlE[1], sy, 0, ps[r][1]);
                    }
                    if (sz[r] >= 0) {
                        xb = stretch_p(xb, p.pmlE[2], sz[r], 0, ps[r][2]);
                        ya = stretch_p(ya, p.pmlE[2], sz[r], 0, ps[r][3]);
                    }
                    if (sx >= 0) {
                        yb = stretch_p(yb, p.pmlE[0], sx, 1, ps[r][4]);
                        za = stretch_p(za, p.pmlE[0], sx, 1, ps[r][5]);
                    }
                    psi_store_p(p.psiE, pc, (unsigned)k, plane, col, sx, sy, sz[r], ps[r]);
                    float2 dxv = p_sub(xa, xb), dyv = p_sub(ya, yb), dzv = p_sub(za, zb);
                    if (src0 || src1) {
                        dxv = p_add(dxv, f2(src0 ? point_drive(p, x, y, k, 0, n) : 0.f, src1 ? point_drive(p, x + 1, y, k, 0, n) : 0.f));
                        dyv = p_add(dyv, f2(src0 ? point_drive(p, x, y, k, 1, n) : 0.f, src1 ? point_drive(p, x + 1, y, k, 1, n) : 0.f));
                        dzv = p_add(dzv, f2(src0 ? point_drive(p, x, y, k, 2, n) : 0.f, src1 ? point_drive(p, x + 1, y, k, 2, n) : 0.f));
                    }
                    ex = p_fma(ca[0], e0[r][0], p_mul(cb[0], dxv));
                    ey = p_fma(ca[1], e0[r][1], p_mul(cb[1], dyv));
                    ez = p_fma(ca[2], e0[r][2], p_mul(cb[2], dzv));
                    // PEC walls: components tangential to a wall at index 0 stay zero (x > 0 holds for x + 1)
                    const bool jm = y > 0, km = k > 0, im = x > 0;
                    if (!(jm && km)) ex = e0[r][0];
                    if (!km) ey = e0[r][1];
                    else if (!im) ey.x = e0[r][1].x;
                    if (!jm) ez = e0[r][2];
                    else if (!im) ez.x = e0[r][2].x;
                }
                if (on0[r] && on1[r]) {
                    stp(p.En[0] + id, ex);
                    stp(p.En[1] + id, ey);
                    stp(p.En[2] + id, ez);
                } else if (on0[r]) {
                    p.En[0][id] = ex.x;
                    p.En[1][id] = ey.x;
                    p.En[2][id] = ez.x;
                    ex.y = ey.y = ez.y = 0.f;
                } else {
                    p.En[0][id + 1] = ex.y;
                    p.En[1][id + 1] = ey.y;
                    p.En[2][id + 1] = ez.y;
                    ex.x = ey.x = ez.x = 0.f;
                }
                if (check)
                    emax = fmaxf(emax, fmaxf(fabsf(ex.x) + fabsf(ey.x) + fabsf(ez.x), fabsf(ex.y) + fabsf(ey.y) + fabsf(ez.y)));
            }
            hxb = h[P - 1][0];   // read only when plane kb + P is this thread's
            hyb = h[P - 1][1];
        }
        if (!(emax < p.blowup)) atomicOr(p.ctl + 2, 1);
    }
    finish_step(p.ctl, p.nblocks_e, n);
}

}  // namespace fdtd
