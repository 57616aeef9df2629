// Design-E kernel on x-adjacent sample pairs (FP32): the E update inside the design box of Eqs.
// (Maxwells)a,b with (eps_mixed), (sigma_mixed), (Poles_mixed) and the pole recursion, as in
// e_design_column, with each thread updating the samples of component C at (i, j, k) and (i+1, j, k):
// 8-byte loads and stores of fields, densities and snapshots, 16-byte loads and stores of the two
// samples' pole currents, and Blackwell's paired FP32 instructions.  Pairs that need a per-sample
// treatment (a gap sample, a point source, the TF/SF plane, a PEC wall, a sample outside its
// component's sample box) and the per-sample records of paper mode take e_design_column sample by sample.
//
// Used when nx and the working box's x origin and extent are even (the host checks), so that a pair's two
// samples are adjacent, and 8-byte aligned, in every array (the density too, in either layout).
#pragma once
#include "fdtd_shell2.cuh"

namespace fdtd {

// L2 prefetch of the rows of the plane FDTD_ED2_PF ahead (0: none); measured 0.0718 -> 0.0699 ms on the
// config-2 design box (3 poles), 0.697 -> 0.653 ms on the config-3 one (6 poles, two blocks per SM)
#ifndef FDTD_ED2_PF
#define FDTD_ED2_PF 1
#endif

__device__ __forceinline__ float4 ldq(const cpx<float>* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void stq(cpx<float>* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

template <int MP, int C>
__device__ __forceinline__ float design_pair_column(const KParams<float>& p, const PoleTable<float>& tab, int i, int j,
                                                    int k0, int k1, int n)
{
    constexpr int ca = C == 0 ? 2 : C - 1, cb = C == 2 ? 0 : C + 1;
    constexpr int MQ = MP > 0 ? MP : 1;
    const float* __restrict__ Ha = p.Hn[ca];
    const float* __restrict__ Hb = p.Hn[cb];
    const float* __restrict__ Ec = p.E[C];
    const float* __restrict__ rc = p.rhoc[C];
    const unsigned nx = (unsigned)p.nx, plane = (unsigned)p.plane, col = (unsigned)j * nx + (unsigned)i;
    const long long dcol = (long long)(j - p.db[2]) * p.dnx + (i - p.db[0]);
    const bool inxy_g = i + 1 >= p.gb[0] && i < p.gb[1] && j >= p.gb[2] && j < p.gb[3];   // either sample
    // per-sample cases for the whole column: paper-mode records, either sample outside the component's
    // sample box in x or y, the TF/SF plane (E_z at x = i0), the PEC walls at x = 0 (C = 1, 2), y = 0 (C = 0, 2)
    const bool col_scalar = p.td_acc || p.hist_dq || i < p.mb[C][0] || i + 1 >= p.mb[C][1] || j < p.mb[C][2] ||
                            j >= p.mb[C][3] || (C == 2 && (i == p.tfsf_i0 || i + 1 == p.tfsf_i0)) ||
                            ((C == 1 || C == 2) && i == 0) || (C != 1 && j == 0);
    const long long slot0 = (long long)((n - p.snap0) % p.K) * 3 * p.nd + C * p.nd;
    const int P = p.P[C], P1 = p.P1[C];
    const float2 idx2 = f2(p.inv_dx, p.inv_dx), one2 = f2(1.f, 1.f);
    const float2 D1 = f2(p.D1[C], p.D1[C]), dD = f2(p.dD[C], p.dD[C]), N1 = f2(p.N1[C], p.N1[C]),
                 dN = f2(p.dN[C], p.dN[C]), hg = f2(p.hg, p.hg);
    float emax = 0.f;
    for (int k = k0; k < k1; ++k) {
        const bool in_gz = k >= p.gb[4] && k < p.gb[5];
        const bool src = p.nb > 0 && k >= p.sb[4] && k < p.sb[5] && j >= p.sb[2] && j < p.sb[3] && i + 1 >= p.sb[0] &&
                         i < p.sb[1];
        // per-sample cases of this plane: a gap sample, a point source, the z range of the sample box, the
        // PEC wall at z = 0 (C = 0, 1)
        if (col_scalar || src || (in_gz && inxy_g) || k < p.mb[C][4] || k >= p.mb[C][5] || (C != 2 && k == 0)) {
#pragma unroll 1
            for (int e = 0; e < 2; ++e) emax = fmaxf(emax, e_design_column<float, MP, C>(p, tab, i + e, j, k, k + 1, n));
            continue;
        }
        const unsigned id = (unsigned)k * plane + col;
        const long long dv = (long long)(k - p.db[4]) * p.dplane + dcol;
        if (FDTD_ED2_PF > 0 && k + FDTD_ED2_PF < k1) {   // the rows of a coming plane into L2
            const unsigned ip = id + FDTD_ED2_PF * plane;
            const long long dp = dv + FDTD_ED2_PF * p.dplane;
            pf_l2(Ha + ip);
            pf_l2(Hb + ip);
            pf_l2(Ec + ip);
            pf_l2(rc + dp);
#pragma unroll
            for (int pp = 0; pp < MQ; ++pp)
                if (pp < P) pf_l2(reinterpret_cast<const float*>(p.Q[C] + pp * p.nd + dp));
        }
        // (curl H)_C = (Ha - Ha(-1 along la)) - (Hb - Hb(-1 along lb)); along x the pair's lower neighbour is
        // its first sample's
        const float2 ha = ldp(Ha + id), hb = ldp(Hb + id);
        float2 ham, hbm;
        if (C == 0) {
            ham = ldp(Ha + id - nx);       // H_z along y
            hbm = ldp(Hb + id - plane);    // H_y along z
        } else if (C == 1) {
            ham = ldp(Ha + id - plane);    // H_x along z
            hbm = f2(Hb[id - 1], hb.x);    // H_z along x
        } else {
            ham = f2(Ha[id - 1], ha.x);    // H_y along x
            hbm = ldp(Hb + id - nx);       // H_x along y
        }
        const float2 e0 = ldp(Ec + id), rho = ldp(rc + dv);
        float4 q[MQ];
#pragma unroll
        for (int pp = 0; pp < MQ; ++pp)
            if (pp < P) q[pp] = ldq(p.Q[C] + pp * p.nd + dv);
        // drive and the blended update, per element the operations of design_update
        const float2 d = p_mul(p_sub(p_sub(ha, ham), p_sub(hb, hbm)), idx2);
        const float2 gm = p_mul(p_mul(hg, rho), p_sub(one2, rho));
        const float2 D = p_add(p_fma(rho, dD, D1), gm);
        const float2 N = p_sub(p_fma(rho, dN, N1), gm);
        float2 sq = f2(0.f, 0.f);
#pragma unroll
        for (int pp = 0; pp < MQ; ++pp) {
            if (pp < P) {
                const float2 kap = pp < P1 ? p_sub(one2, rho) : rho;
                const cpx<float> g = tab.g[C][pp];
                const float2 qre = f2(q[pp].x, q[pp].z), qim = f2(q[pp].y, q[pp].w);
                sq = p_fma(kap, p_sub(p_mul(f2(g.re, g.re), qre), p_mul(f2(g.im, g.im), qim)), sq);
            }
        }
        const float2 num = p_sub(p_fma(N, e0, d), sq);
        const float2 e = f2(div_t(num.x, D.x), div_t(num.y, D.y));
        const float2 es = p_add(e, e0);
#pragma unroll
        for (int pp = 0; pp < MQ; ++pp) {
            if (pp < P) {
                const cpx<float> a = tab.am1[C][pp], b = tab.beta[C][pp];
                const float2 qre = f2(q[pp].x, q[pp].z), qim = f2(q[pp].y, q[pp].w);
                const float2 vre = p_fma(f2(b.re, b.re), es, p_add(qre, p_sub(p_mul(f2(a.re, a.re), qre), p_mul(f2(a.im, a.im), qim))));
                const float2 vim = p_fma(f2(b.im, b.im), es, p_add(qim, p_fma(f2(a.re, a.re), qim, p_mul(f2(a.im, a.im), qre))));
                stq(p.Q[C] + pp * p.nd + dv, make_float4(vre.x, vim.x, vre.y, vim.y));
            }
        }
        stp(p.En[C] + id, e);
        stp(p.snap + slot0 + dv, e);
        emax = fmaxf(emax, fmaxf(fabsf(e.x), fabsf(e.y)));
    }
    return emax;
}

// Resident blocks per SM the register allocation is held to (the pole currents of a pair take twice
// the registers of a sample's).
template <int MP>
constexpr int ed2_min_blocks()
{
#ifdef FDTD_ED2_MINB
    return FDTD_ED2_MINB;
#else
    return MP <= 4 ? 4 : 2;   // MP <= 8
#endif
}

// One block: 32 x 8 threads over 64 x 8 (x, y) samples of component blockIdx.z % 3, a column of p.edz planes.
template <int MP>
__global__ void __launch_bounds__(kBX * kBY, ed2_min_blocks<MP>()) e_design2_kernel(const KParams<float> p,
                                                                                         const PoleTable<float> tab)
{
    const int zc = blockIdx.z / 3, c = blockIdx.z - 3 * zc;
    const int i = p.db[0] + 2 * (blockIdx.x * kBX + threadIdx.x);
    const int j = p.db[2] + blockIdx.y * kBY + threadIdx.y;
    const int k0 = p.db[4] + zc * p.edz, k1 = min(p.db[5], k0 + p.edz);
    pdl_wait();
    pdl_trigger();
    const int n = read_step<float>(p.ctl);
    if (i < p.db[1] && j < p.db[3]) {
        const float emax = c == 0 ? design_pair_column<MP, 0>(p, tab, i, j, k0, k1, n)
                         : c == 1 ? design_pair_column<MP, 1>(p, tab, i, j, k0, k1, n)
                                  : design_pair_column<MP, 2>(p, tab, i, j, k0, k1, n);
        if (!(emax < p.blowup)) atomicOr(p.ctl + 2, 1);
    }
    finish_step(p.ctl, p.nblocks_e, n);
}

}  // namespace fdtd
