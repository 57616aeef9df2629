// Background step for sm_103a: H^{n+1/2} everywhere and E^{n+1} for every cell outside the design
// box (Yee update of Eqs. (Maxwells)a-c with the background material, CFS-CPML psi in the edge slabs,
// the TF/SF correction and point sources), reading E^n / H^{n-1/2} from one buffer of each pair and
// writing the other.  The grid is split in two:
//
// * an interior box of tiles (the last column or row may be partial), away from the walls and the CPML
//   slabs, updated by step_kernel in one pass: 48 B per cell (each field word read once and written
//   once) instead of the 72 B of separate H and E passes.  A block owns a kTX x kTY tile and marches
//   through p.kc (at most kKC) z planes (plus the
//   plane below, whose H is the z-1 neighbour of the first E update); each thread updates two
//   x-adjacent cells with paired FP32 arithmetic (one instruction for both cells) and 8-byte shared /
//   global accesses.  Per plane, TMA brings E^n and H^{n-1/2} of the tile plus a one-cell halo into
//   shared-memory rings NE / NH planes ahead of use; H^{n+1/2} is computed on the tile and on its
//   -x/-y halo and stored; after one barrier the producer thread refills the plane's ring slots and
//   E^{n+1} follows from the shared H and the plane below, kept in registers.  Tiles touched by the
//   TF/SF plane, a point source or the design-box rim take a path with per-cell tests;
// * the shell around it (walls, CPML slabs, ragged edges), updated column by column by
//   shell_h_kernel (H) and then shell_e_kernel (E, after every H of the step is stored).
//
// A halo H value the interior kernel recomputes is bit-identical to the one the shell or another
// block stores: the formula depends only on the cell and every operation is explicitly rounded.
// Every mbarrier wait is bounded: on a timeout the block sets ctl[2] bit 2, drains the copies it
// issued (again bounded) and leaves.
#pragma once
#include <climits>

#include "fdtd_kernels.cuh"

namespace fdtd {

static_assert(kKC + 1 <= 32, "per-plane path table holds 32 planes");

// ---- explicitly rounded scalar and paired arithmetic -------------------------------------------
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
struct Pair;
template <>
struct Pair<float> {
    using V = float2;
};
template <>
struct Pair<double> {
    using V = double2;
};

// Per component identical to the scalar _rn operations above (a - b = fma(b, -1, a), one rounding).
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 p_sub(double2 a, double2 b) { return make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y)); }
__device__ __forceinline__ double2 p_fma(double2 a, double2 b, double2 c)
{
    return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 p_mul(double2 a, double2 b) { return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)); }

template <typename V, typename T>
__device__ __forceinline__ V pv(T a, T b)
{
    V v;
    v.x = a;
    v.y = b;
    return v;
}
template <typename V>
__device__ __forceinline__ auto el(const V& v, int c) -> decltype(v.x)
{
    return c ? v.y : v.x;
}
template <typename V, typename T>
__device__ __forceinline__ void set_el(V& v, int c, T a)
{
    if (c)
        v.y = a;
    else
        v.x = a;
}
template <typename V, typename T>
__device__ __forceinline__ V ld2(const T* s)
{
    return *reinterpret_cast<const V*>(s);
}
template <typename V, typename T>
__device__ __forceinline__ void st2(T* d, const V& v)
{
    *reinterpret_cast<V*>(d) = v;
}

// ---- TMA and mbarrier ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// 4-D tiled TMA load (x, y, z, component) into shared memory, completing on an mbarrier.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z, int c)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
            smem_addr(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(c), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long kWaitNs = 50ull * 1000 * 1000;   // a TMA plane arrives in microseconds

// Wait for the phase of the given parity; false after limit_ns (or 2^26 tries) without completion.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned long long limit_ns = kWaitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (int t = 0; t < (1 << 26); ++t) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// ---- per-cell update rules ---------------------------------------------------------------------
// Staged neighbourhood of one cell for the H update: E^n at the cell, at y+1, x+1, z+1; H^{n-1/2}.
template <typename T>
struct HIn {
    T ex0, ey0, ez0, ezy, exy, ezx, eyx, exz, eyz, hox, hoy, hoz;
};

// H^{n+1/2} of a cell outside every slab: H = Ho + cneg ((a - b) - (c - d)), cneg = -(dt/mu0)/dx,
// the TF/SF correction in the x difference of H_y.  tf: the cell is the one left of the TF/SF plane.
template <typename T>
__device__ __forceinline__ void h_cheap(const HIn<T>& a, T cneg, bool tf, T einc_n, T& hx, T& hy, T& hz)
{
    const T dyx = tf ? sub_rn(sub_rn(a.ezx, a.ez0), einc_n) : sub_rn(a.ezx, a.ez0);
    hx = fma_rn(cneg, sub_rn(sub_rn(a.ezy, a.ez0), sub_rn(a.eyz, a.ey0)), a.hox);
    hy = fma_rn(cneg, sub_rn(sub_rn(a.exz, a.ex0), dyx), a.hoy);
    hz = fma_rn(cneg, sub_rn(sub_rn(a.eyx, a.ey0), sub_rn(a.exy, a.ex0)), a.hoz);
}

// E^{n+1} of one cell from the six H differences (unscaled) and E^n.  Cells outside the slabs, off
// the walls and outside the source box take E = ca E + (cb/dx)((a - b) - (c - d)); the others scale
// each difference by 1/dx, stretch the slab terms (psi_E in place), add the point-source drive and
// keep the wall-tangential components at zero.
template <typename T>
struct EOut {
    T ex, ey, ez;
};

template <typename T>
__device__ __forceinline__ EOut<T> e_cell(const KParams<T>& p, int i, int j, int k, int n, T hinc_n, T ex0, T ey0, T ez0,
                                          T rxa, T rxb, T rya, T ryb, T rza, T rzb)
{
    const bool tf = i == p.tfsf_i0;                                        // H_y(i0-1/2) is scattered field
    const int sx = slab_index(i, p.cpl[0], p.cph[0], p.nx);
    const int sy = slab_index(j, p.cpl[1], p.cph[1], p.ny);
    const int sz = slab_index(k, p.cpl[2], p.cph[2], p.nz);
    const bool src = p.nb > 0 && in_box(p.sb, i, j, k);
    EOut<T> e;
    if (sx < 0 && sy < 0 && sz < 0 && !src && i > 0 && j > 0 && k > 0) {
        e.ex = p.bg_ca[0] * ex0 + p.bg_cbi[0] * (rxa - rxb);
        e.ey = p.bg_ca[1] * ey0 + p.bg_cbi[1] * (rya - ryb);
        e.ez = p.bg_ca[2] * ez0 + p.bg_cbi[2] * ((tf ? rza - hinc_n : rza) - rzb);
        return e;
    }
    const T idx = p.inv_dx;
    T xa = rxa * idx, xb = rxb * idx, ya = rya * idx, yb = ryb * idx, za = rza * idx, zb = rzb * idx;
    if (tf) za -= hinc_n * idx;
    if (sy >= 0) {
        const long long q = psi_index(p, i, j, k, 1, sy);
        xa = stretch(xa, p.pmlE[1], sy, p.psiE[0][0] + q);
        zb = stretch(zb, p.pmlE[1], sy, p.psiE[2][1] + q);
    }
    if (sz >= 0) {
        const long long q = psi_index(p, i, j, k, 2, sz);
        xb = stretch(xb, p.pmlE[2], sz, p.psiE[0][1] + q);
        ya = stretch(ya, p.pmlE[2], sz, p.psiE[1][0] + q);
    }
    if (sx >= 0) {
        const long long q = psi_index(p, i, j, k, 0, sx);
        yb = stretch(yb, p.pmlE[0], sx, p.psiE[1][1] + q);
        za = stretch(za, p.pmlE[0], sx, p.psiE[2][0] + q);
    }
    T dxv = xa - xb, dyv = ya - yb, dzv = za - zb;
    if (src) {
        dxv += point_drive(p, i, j, k, 0, n);
        dyv += point_drive(p, i, j, k, 1, n);
        dzv += point_drive(p, i, j, k, 2, n);
    }
    e.ex = p.bg_ca[0] * ex0 + p.bg_cb[0] * dxv;
    e.ey = p.bg_ca[1] * ey0 + p.bg_cb[1] * dyv;
    e.ez = p.bg_ca[2] * ez0 + p.bg_cb[2] * dzv;
    const bool im = i > 0, jm = j > 0, km = k > 0;
    if (!(jm && km)) e.ex = ex0;   // PEC walls: components tangential to a wall at index 0 stay zero
    if (!(km && im)) e.ey = ey0;
    if (!(im && jm)) e.ez = ez0;
    return e;
}

// ---- interior: fused TMA kernel -----------------------------------------------------------------
// H^{n+1/2} of one interior cell (scalar; the -x halo column) at staged offset o = ey * kSX + ex.
template <typename T>
__device__ __forceinline__ void h_one(const KParams<T>& p, const T* E0, const T* E1, const T* Ho, int o, int x, T cneg,
                                      T einc_n, T& hx, T& hy, T& hz)
{
    constexpr int PE = kSYE * kSX, PH = kSYH * kSX;
    HIn<T> a;
    a.ex0 = E0[o];
    a.ey0 = E0[PE + o];
    a.ez0 = E0[2 * PE + o];
    a.ezy = E0[2 * PE + o + kSX];
    a.exy = E0[o + kSX];
    a.ezx = E0[2 * PE + o + 1];
    a.eyx = E0[PE + o + 1];
    a.exz = E1[o];
    a.eyz = E1[PE + o];
    a.hox = Ho[o];
    a.hoy = Ho[PH + o];
    a.hoz = Ho[2 * PH + o];
    h_cheap(a, cneg, x == p.tfsf_i0 - 1, einc_n, hx, hy, hz);
}

// H^{n+1/2} of the interior cell pair (x, x+1) at staged offset o (even); e0 returns the pair's E^n.
// Per component the same operations as h_cheap.  TF: the tile holds the TF/SF plane.
template <typename T, bool TF>
__device__ __forceinline__ void h_pair(const KParams<T>& p, const T* E0, const T* E1, const T* Ho, int o, int x, T cneg,
                                       T einc_n, typename Pair<T>::V (&e0)[3], typename Pair<T>::V (&h)[3])
{
    using V = typename Pair<T>::V;
    constexpr int PE = kSYE * kSX, PH = kSYH * kSX;
    e0[0] = ld2<V>(E0 + o);
    e0[1] = ld2<V>(E0 + PE + o);
    e0[2] = ld2<V>(E0 + 2 * PE + o);
    const V ezy = ld2<V>(E0 + 2 * PE + o + kSX), exy = ld2<V>(E0 + o + kSX);
    const V ezn = ld2<V>(E0 + 2 * PE + o + 2), eyn = ld2<V>(E0 + PE + o + 2);
    const V ezx = pv<V>(e0[2].y, ezn.x), eyx = pv<V>(e0[1].y, eyn.x);
    const V exz = ld2<V>(E1 + o), eyz = ld2<V>(E1 + PE + o);
    const V hox = ld2<V>(Ho + o), hoy = ld2<V>(Ho + PH + o), hoz = ld2<V>(Ho + 2 * PH + o);
    const V cn = pv<V>(cneg, cneg);
    V dyx = p_sub(ezx, e0[2]);
    if (TF && p.tfsf_i0 - 1 >= x && p.tfsf_i0 - 1 <= x + 1)   // subtracting +0 from the other cell is exact
        dyx = p_sub(dyx, pv<V>(x == p.tfsf_i0 - 1 ? einc_n : T(0), x + 1 == p.tfsf_i0 - 1 ? einc_n : T(0)));
    h[0] = p_fma(cn, p_sub(p_sub(ezy, e0[2]), p_sub(eyz, e0[1])), hox);
    h[1] = p_fma(cn, p_sub(p_sub(exz, e0[0]), dyx), hoy);
    h[2] = p_fma(cn, p_sub(p_sub(eyx, e0[1]), p_sub(exy, e0[0])), hoz);
}

// E phase of the own pair: E^{n+1} from its H (registers), the -x / -y neighbours (sHc) and the
// plane below (hxp, hyp).  LITE: per-cell tests for the TF/SF plane, point sources and the design-box
// rim (eup 2); eup 0: the tile is inside the design box (no E update here).
template <typename T, bool LITE>
__device__ __forceinline__ void e_pair(const KParams<T>& p, const T* sHc, int on, int i, int j, int k, int n, int eup,
                                       T hinc_n, const typename Pair<T>::V (&e0)[3], const typename Pair<T>::V (&h)[3],
                                       const typename Pair<T>::V& hxp, const typename Pair<T>::V& hyp, long long id,
                                       bool check, T& emax)
{
    using V = typename Pair<T>::V;
    constexpr int PN = kSYH * kHW;
    if (eup == 0) return;
    const V hzy = ld2<V>(sHc + 2 * PN + on - kHW), hxy = ld2<V>(sHc + on - kHW);      // y - 1
    const V hzl = ld2<V>(sHc + 2 * PN + on - 2), hyl = ld2<V>(sHc + PN + on - 2);    // pair at x - 2
    const V hzx = pv<V>(hzl.y, h[2].x), hyx = pv<V>(hyl.y, h[1].x);                   // x - 1
    const V rxa = p_sub(h[2], hzy), rxb = p_sub(h[1], hyp);
    const V rya = p_sub(h[0], hxp), ryb = p_sub(h[2], hzx);
    const V rza = p_sub(h[1], hyx), rzb = p_sub(h[0], hxy);
    if (!LITE) {
        const V ex = p_fma(pv<V>(p.bg_ca[0], p.bg_ca[0]), e0[0], p_mul(pv<V>(p.bg_cbi[0], p.bg_cbi[0]), p_sub(rxa, rxb)));
        const V ey = p_fma(pv<V>(p.bg_ca[1], p.bg_ca[1]), e0[1], p_mul(pv<V>(p.bg_cbi[1], p.bg_cbi[1]), p_sub(rya, ryb)));
        const V ez = p_fma(pv<V>(p.bg_ca[2], p.bg_ca[2]), e0[2], p_mul(pv<V>(p.bg_cbi[2], p.bg_cbi[2]), p_sub(rza, rzb)));
        st2(p.En[0] + id, ex);
        st2(p.En[1] + id, ey);
        st2(p.En[2] + id, ez);
        if (check) emax = fmax(emax, fmax(fabs(ex.x) + fabs(ey.x) + fabs(ez.x), fabs(ex.y) + fabs(ey.y) + fabs(ez.y)));
        return;
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int ic = i + c;
        if (eup == 2 && in_box(p.db, ic, j, k)) continue;
        const EOut<T> e = e_cell(p, ic, j, k, n, hinc_n, el(e0[0], c), el(e0[1], c), el(e0[2], c), el(rxa, c), el(rxb, c),
                                 el(rya, c), el(ryb, c), el(rza, c), el(rzb, c));
        p.En[0][id + c] = e.ex;
        p.En[1][id + c] = e.ey;
        p.En[2][id + c] = e.ez;
        if (check) emax = fmax(emax, fabs(e.ex) + fabs(e.ey) + fabs(e.ez));
    }
}

// Path of each plane of the block's chunk: bit 0 lite (else plain), bits 1-2 eup: 0 no E update
// (tile inside the design box), 1 every cell, 2 per-cell design-box test.
template <typename T>
__device__ __forceinline__ int plane_path(const KParams<T>& p, int i0, int j0, int k)
{
    const bool dz = k >= p.db[4] && k < p.db[5];
    const bool db_any = p.db[0] < i0 + kTX && p.db[1] > i0 && p.db[2] < j0 + kTY && p.db[3] > j0;
    const bool db_all = p.db[0] <= i0 && p.db[1] >= i0 + kTX && p.db[2] <= j0 && p.db[3] >= j0 + kTY;
    const int eup = (dz && db_all) ? 0 : ((dz && db_any) ? 2 : 1);
    const bool src = p.nb > 0 && p.sb[0] < i0 + kTX && p.sb[1] > i0 && p.sb[2] < j0 + kTY && p.sb[3] > j0 &&
                     k >= p.sb[4] && k < p.sb[5];
    const bool tf = p.tfsf_i0 >= i0 && p.tfsf_i0 <= i0 + kTX;
    return ((eup == 2 || src || tf) ? 1 : 0) | (eup << 1);
}

template <typename T>
__global__ void __launch_bounds__(kPX * kTY, StepCfg<T>::MINB)
    step_kernel(const __grid_constant__ KParams<T> p, const __grid_constant__ StepMaps m)
{
    using V = typename Pair<T>::V;
    constexpr int NE = StepCfg<T>::NE, NH = StepCfg<T>::NH;
    constexpr int PN = kSYH * kHW;    // one component of a new-H tile
    using S = StepSmem<T>;
    static_assert((NE + NH + 1) * sizeof(uint64_t) <= S::bars, "mbarriers of the rings and the test hook");
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    T* sE = (T*)sm;                                                    // NE slots of S::e_slot bytes
    T* sHo = (T*)(sm + NE * S::e_slot);                                // NH slots of S::h_slot bytes
    T* sHn = (T*)(sm + NE * S::e_slot + NH * S::h_slot);               // two new-H tiles, by plane parity
    int* path = (int*)(sm + NE * S::e_slot + NH * S::h_slot + S::h_new);
    uint64_t* bar = (uint64_t*)(sm + NE * S::e_slot + NH * S::h_slot + S::h_new + S::table);   // [NE] E, [NH] H
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kPX + tx;
    const int i0 = p.ib[0] + blockIdx.x * kTX, j0 = p.ib[2] + blockIdx.y * kTY;
    const int i = i0 + 2 * tx, j = j0 + ty;                            // first cell of the own pair
    // the last tile column and row may be partial: cells beyond the box are the shell's (their H is
    // computed here too, for nothing, but neither stored nor used by a cell of the box)
    const bool own = i < p.ib[1] && j < p.ib[3];
    const int kb = p.ib[4] + blockIdx.z * p.kc, ke = min(kb + p.kc, p.ib[5]);
    const int k_first = kb - 1;            // >= 0: the interior box starts above plane 0
    const int ne_tot = ke - k_first + 1;   // E planes k_first .. ke
    const int nh_tot = ke - k_first;       // H planes k_first .. ke-1
    pdl_wait();
    pdl_trigger();
    const int n = read_step<T>(p.ctl);
    auto eslot = [&](int s) { return (T*)((unsigned char*)sE + s * S::e_slot); };
    auto hslot = [&](int s) { return (T*)((unsigned char*)sHo + s * S::h_slot); };
    auto issue_e = [&](int r) {
        mbar_expect_tx(bar + r % NE, S::e_tx);
        tma_load_4d(eslot(r % NE), &m.e, bar + r % NE, i0 - kOX, j0 - 1, k_first + r, 0);
    };
    auto issue_h = [&](int r) {
        mbar_expect_tx(bar + NE + r % NH, S::h_tx);
        tma_load_4d(hslot(r % NH), &m.h, bar + NE + r % NH, i0 - kOX, j0 - 1, k_first + r, 0);
    };
    if (tid == 0) {
        for (int s = 0; s < NE + NH + 1; ++s) mbar_init(bar + s, 1);   // [NE + NH]: the test hook's barrier
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_shared();
    }
    if (tid < nh_tot) path[tid] = plane_path(p, i0, j0, k_first + tid);
    // a block that starts after another one timed out does nothing (the run is already failed)
    const bool skip = __syncthreads_or(tid == 0 && (__ldcg(p.ctl + 2) & 4));
    int e_issued = 0, h_issued = 0;        // meaningful in thread 0
    if (tid == 0 && !skip) {
        for (; e_issued < NE && e_issued < ne_tot; ++e_issued) issue_e(e_issued);
        for (; h_issued < NH && h_issued < nh_tot; ++h_issued) issue_h(h_issued);
    }
    const T cneg = -(p.ch * p.inv_dx);
    const T einc_n = p.tfsf_i0 >= 0 ? __ldg(p.einc + n) : T(0);
    const T hinc_n = p.tfsf_i0 >= 0 ? __ldg(p.hinc + n) : T(0);
    const bool check = (n & 15) == 0 || n + 1 == p.n_steps;   // blow-up test on every 16th and the last step
    const int o = (ty + 1) * kSX + kOX + 2 * tx;       // own pair in a staged plane
    const int on = (ty + 1) * kHW + 2 + 2 * tx;        // own pair in a new-H tile
    V hxp = pv<V>(T(0), T(0)), hyp = hxp;              // H of the own pair on the plane below
    V e0[3], h[3];
    T emax = T(0);
    long long id = ((long long)k_first * p.ny + j) * p.nx + i;   // own pair of the plane (stores for k >= kb)
    int es = 0, hs = 0;                                          // ring slots of E plane r and H plane r
    bool failed = false;
    for (int r = 0; r < (skip ? 0 : nh_tot); ++r) {
        const int k = k_first + r;
        const int es1 = es + 1 == NE ? 0 : es + 1;
        bool ok = true;
        if (r == 0) ok = mbar_wait(bar, 0);
        // failure-path test hook: a wait on a barrier that no copy completes runs out after stall_ns
        if (r == 0 && p.stall_ns > 0 && n == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)
            ok = mbar_wait(bar + NE + NH, 0, (unsigned long long)p.stall_ns) && ok;
        ok = ok && mbar_wait(bar + es1, ((r + 1) / NE) & 1);
        ok = ok && mbar_wait(bar + NE + hs, (r / NH) & 1);
        const int pa = path[r];
        const bool lite = pa & 1;
        const int eup = pa >> 1;
        const T* E0 = eslot(es);
        const T* E1 = eslot(es1);
        const T* Ho = hslot(hs);
        T* sHc = sHn + (r & 1) * 3 * PN;
        if (lite)
            h_pair<T, true>(p, E0, E1, Ho, o, i, cneg, einc_n, e0, h);
        else
            h_pair<T, false>(p, E0, E1, Ho, o, i, cneg, einc_n, e0, h);
        if (r > 0) {
            st2(sHc + on, h[0]);
            st2(sHc + PN + on, h[1]);
            st2(sHc + 2 * PN + on, h[2]);
            if (own) {
                st2(p.Hn[0] + id, h[0]);
                st2(p.Hn[1] + id, h[1]);
                st2(p.Hn[2] + id, h[2]);
            }
            // halo work goes to three different warps (the second half of warps 7, 6 and 5), so that
            // no warp carries more than one extra cell update per plane
            if (ty == kTY - 1) {                           // -y halo row, as pairs
                V eh[3], hh[3];
                if (lite)
                    h_pair<T, true>(p, E0, E1, Ho, kOX + 2 * tx, i, cneg, einc_n, eh, hh);
                else
                    h_pair<T, false>(p, E0, E1, Ho, kOX + 2 * tx, i, cneg, einc_n, eh, hh);
                st2(sHc + 2 + 2 * tx, hh[0]);
                st2(sHc + PN + 2 + 2 * tx, hh[1]);
                st2(sHc + 2 * PN + 2 + 2 * tx, hh[2]);
            } else if (ty == kTY - 3 || (ty == kTY - 5 && tx == 0)) {   // -x halo column: rows j0.., the corner
                const int ly = ty == kTY - 3 ? tx + 1 : 0;
                T a, b, c;
                h_one(p, E0, E1, Ho, ly * kSX + kOX - 1, i0 - 1, cneg, einc_n, a, b, c);
                sHc[ly * kHW + 1] = a;
                sHc[PN + ly * kHW + 1] = b;
                sHc[2 * PN + ly * kHW + 1] = c;
            }
        }
        if (__syncthreads_or(!ok)) {       // the new-H tile is complete; plane r's ring slots are free
            failed = true;
            break;
        }
        if (tid == 0) {
            fence_async_shared();
            if (e_issued < ne_tot) issue_e(e_issued++);
            if (h_issued < nh_tot) issue_h(h_issued++);
        }
        if (r > 0 && own) {
            if (lite)
                e_pair<T, true>(p, sHc, on, i, j, k, n, eup, hinc_n, e0, h, hxp, hyp, id, check, emax);
            else
                e_pair<T, false>(p, sHc, on, i, j, k, n, eup, hinc_n, e0, h, hxp, hyp, id, check, emax);
        }
        hxp = h[0];
        hyp = h[1];
        id += p.plane;
        es = es1;
        hs = hs + 1 == NH ? 0 : hs + 1;
    }
    if (failed) {
        if (tid == 0) {
            atomicOr(p.ctl + 2, 4);
            // drain every copy this block issued before leaving (bounded)
            for (int r = 0; r < e_issued; ++r) mbar_wait(bar + r % NE, (r / NE) & 1);
            for (int r = 0; r < h_issued; ++r) mbar_wait(bar + NE + r % NH, (r / NH) & 1);
        }
        __syncthreads();
    }
    if (!(emax < p.blowup)) atomicOr(p.ctl + 2, 1);
}

// ---- shell: per-cell kernels ----------------------------------------------------------------------
// Block b -> box q; a block covers kShellCells consecutive (x, y) columns of the box (x fastest, so a
// warp reads and writes consecutive addresses even in boxes narrower than a warp), and each thread
// marches s.kz (at most kShellKZ) planes of its column in batches of kShellPZ planes whose loads are all
// issued before any store.  The per-column set-up (box search, column coordinates, slab indices) is
// paid once per s.kz planes; cell and psi offsets are 32-bit (a grid holds fewer than 2^31
// cells) and advance by a fixed stride per plane.
constexpr int kShellCells = kBX * kBY;

struct ShellCol {
    int x, y, k0, k1;   // column, planes [k0, k1)
};

__device__ __forceinline__ bool shell_cell(const ShellBoxes& s, ShellCol& c)
{
    int q = 0;
    while (q + 1 < s.n && blockIdx.x >= s.first[q + 1]) ++q;
    const int* B = s.b[q];
    const unsigned loc = blockIdx.x - s.first[q];
    const unsigned wx = B[1] - B[0], wxy = wx * (B[3] - B[2]);
    const unsigned chunks = (wxy + kShellCells - 1) / kShellCells;
    const unsigned zc = loc / chunks;
    const unsigned t = (loc - zc * chunks) * kShellCells + threadIdx.y * kBX + threadIdx.x;
    const unsigned yy = t / wx;
    c.x = B[0] + (int)(t - yy * wx);
    c.y = B[2] + (int)yy;
    c.k0 = B[4] + (int)zc * s.kz;
    c.k1 = min(B[5], c.k0 + s.kz);
    return t < wxy;
}

// 32-bit psi offsets of one column: x slab ((k ny + y) W0 + sx) = k qxs + qx0, y slab
// ((k W1 + sy) nx + x) = k qys + qy0, z slab ((sz ny + y) nx + x) = sz plane + col.
struct PsiCol {
    unsigned qx0, qxs, qy0, qys;
};

template <typename T>
__device__ __forceinline__ PsiCol psi_col(const KParams<T>& p, int x, int y, int sx, int sy)
{
    PsiCol c;
    c.qxs = (unsigned)p.ny * (unsigned)p.W[0];
    c.qx0 = (unsigned)y * (unsigned)p.W[0] + (unsigned)max(sx, 0);
    c.qys = (unsigned)p.W[1] * (unsigned)p.nx;
    c.qy0 = (unsigned)max(sy, 0) * (unsigned)p.nx + (unsigned)x;
    return c;
}

// psi of one cell for the six curl terms (0 outside the slabs): [0] d/dy of the x row, [1] d/dy of
// the z row (y slab); [2] d/dz of the x row, [3] d/dz of the y row (z slab); [4] d/dx of the y row,
// [5] d/dx of the z row (x slab).
template <typename T, bool CG>
__device__ __forceinline__ void psi_load(T* const (&ps)[3][2], const PsiCol& pc, unsigned k, unsigned plane,
                                         unsigned col, int sx, int sy, int sz, T (&v)[6])
{
    const unsigned q1 = k * pc.qys + pc.qy0, q2 = (unsigned)max(sz, 0) * plane + col, q0 = k * pc.qxs + pc.qx0;
    v[0] = sy >= 0 ? ldf<CG>(ps[0][0] + q1) : T(0);
    v[1] = sy >= 0 ? ldf<CG>(ps[2][1] + q1) : T(0);
    v[2] = sz >= 0 ? ldf<CG>(ps[0][1] + q2) : T(0);
    v[3] = sz >= 0 ? ldf<CG>(ps[1][0] + q2) : T(0);
    v[4] = sx >= 0 ? ldf<CG>(ps[1][1] + q0) : T(0);
    v[5] = sx >= 0 ? ldf<CG>(ps[2][0] + q0) : T(0);
}

template <typename T>
__device__ __forceinline__ void psi_store(T* const (&ps)[3][2], const PsiCol& pc, unsigned k, unsigned plane,
                                          unsigned col, int sx, int sy, int sz, const T (&v)[6])
{
    if (sy >= 0) {
        const unsigned q = k * pc.qys + pc.qy0;
        ps[0][0][q] = v[0];
        ps[2][1][q] = v[1];
    }
    if (sz >= 0) {
        const unsigned q = (unsigned)sz * plane + col;
        ps[0][1][q] = v[2];
        ps[1][0][q] = v[3];
    }
    if (sx >= 0) {
        const unsigned q = k * pc.qxs + pc.qx0;
        ps[1][1][q] = v[4];
        ps[2][0][q] = v[5];
    }
}

// d -> d/kappa + psi', psi' = b psi + c d (psi updated in place).
template <typename T>
__device__ __forceinline__ T stretch_v(T d, const T* __restrict__ tab, int s, T& psi)
{
    T kinv, b, c;
    pml_coef(tab, s, kinv, b, c);
    psi = add_rn(mul_rn(b, psi), mul_rn(c, d));
    return add_rn(mul_rn(d, kinv), psi);
}

// H^{n+1/2} of one column (x, y), planes [k0, k1) (at most kShellKZ of them): every cell update of
// the shell, CPML psi_H included.  Within a batch every load is issued before any store (the buffers
// it writes are not the ones it reads); E_x, E_y of the plane above a batch carry over as the next
// batch's own.  CG: state loads bypass L1 (for a persistent kernel whose earlier work items on the
// same SM may hold stale lines).
template <typename T, bool CG>
__device__ __forceinline__ void h_column(const KParams<T>& p, int x, int y, int k0, int k1, int n)
{
    constexpr int P = kShellPZ;
    const T cneg = -(p.ch * p.inv_dx), idx = p.inv_dx, ch = p.ch;
    const T einc_n = p.tfsf_i0 >= 0 ? __ldg(p.einc + n) : T(0);
    const bool tf = x == p.tfsf_i0 - 1;   // H_y here is scattered field
    const int sx = slab_index(x, p.cpl[0], p.cph[0], p.nx), sy = slab_index(y, p.cpl[1], p.cph[1], p.ny);
    const bool xp = x + 1 < p.nx, yp = y + 1 < p.ny;
    const unsigned nx = (unsigned)p.nx, plane = (unsigned)p.plane, col = (unsigned)y * nx + (unsigned)x;
    const PsiCol pc = psi_col(p, x, y, sx, sy);
    const T* __restrict__ E0 = p.E[0];
    const T* __restrict__ E1 = p.E[1];
    const T* __restrict__ E2 = p.E[2];
    T exc = ldf<CG>(E0 + (unsigned)k0 * plane + col), eyc = ldf<CG>(E1 + (unsigned)k0 * plane + col);
    for (int it = 0; it < kShellKZ / P; ++it) {   // compile-time trip bound; k1 may end the column early
        const int kb = k0 + it * P;
        if (kb >= k1) break;
        HIn<T> a[P];
        T ps[P][6];
        int sz[P];
#pragma unroll
        for (int r = 0; r < P; ++r) {
            const int k = kb + r;
            sz[r] = slab_index(k, p.cpl[2], p.cph[2], p.nz);
            if (k >= k1) continue;
            const unsigned id = (unsigned)k * plane + col;
            const bool zp = k + 1 < p.nz;
            a[r].ex0 = r == 0 ? exc : a[r - 1].exz;
            a[r].ey0 = r == 0 ? eyc : a[r - 1].eyz;
            a[r].ez0 = ldf<CG>(E2 + id);
            a[r].ezy = yp ? ldf<CG>(E2 + id + nx) : T(0);
            a[r].exy = yp ? ldf<CG>(E0 + id + nx) : T(0);
            a[r].ezx = xp ? ldf<CG>(E2 + id + 1) : T(0);
            a[r].eyx = xp ? ldf<CG>(E1 + id + 1) : T(0);
            a[r].exz = zp ? ldf<CG>(E0 + id + plane) : T(0);
            a[r].eyz = zp ? ldf<CG>(E1 + id + plane) : T(0);
            a[r].hox = ldf<CG>(p.H[0] + id);
            a[r].hoy = ldf<CG>(p.H[1] + id);
            a[r].hoz = ldf<CG>(p.H[2] + id);
            psi_load<T, CG>(p.psiH, pc, (unsigned)k, plane, col, sx, sy, sz[r], ps[r]);
        }
#pragma unroll
        for (int r = 0; r < P; ++r) {
            const int k = kb + r;
            if (k >= k1) continue;
            const unsigned id = (unsigned)k * plane + col;
            const HIn<T>& c = a[r];
            T hx, hy, hz;
            if (sx < 0 && sy < 0 && sz[r] < 0) {
                h_cheap(c, cneg, tf, einc_n, hx, hy, hz);
            } else {
                T xa = mul_rn(sub_rn(c.ezy, c.ez0), idx), xb = mul_rn(sub_rn(c.eyz, c.ey0), idx);
                T ya = mul_rn(sub_rn(c.exz, c.ex0), idx), yb = mul_rn(sub_rn(c.ezx, c.ez0), idx);
                T za = mul_rn(sub_rn(c.eyx, c.ey0), idx), zb = mul_rn(sub_rn(c.exy, c.ex0), idx);
                if (tf) yb = sub_rn(yb, mul_rn(einc_n, idx));
                if (sy >= 0) {
                    xa = stretch_v(xa, p.pmlH[1], sy, ps[r][0]);
                    zb = stretch_v(zb, p.pmlH[1], sy, ps[r][1]);
                }
                if (sz[r] >= 0) {
                    xb = stretch_v(xb, p.pmlH[2], sz[r], ps[r][2]);
                    ya = stretch_v(ya, p.pmlH[2], sz[r], ps[r][3]);
                }
                if (sx >= 0) {
                    yb = stretch_v(yb, p.pmlH[0], sx, ps[r][4]);
                    za = stretch_v(za, p.pmlH[0], sx, ps[r][5]);
                }
                hx = sub_rn(c.hox, mul_rn(ch, sub_rn(xa, xb)));
                hy = sub_rn(c.hoy, mul_rn(ch, sub_rn(ya, yb)));
                hz = sub_rn(c.hoz, mul_rn(ch, sub_rn(za, zb)));
                psi_store(p.psiHn, pc, (unsigned)k, plane, col, sx, sy, sz[r], ps[r]);
            }
            p.Hn[0][id] = hx;
            p.Hn[1][id] = hy;
            p.Hn[2][id] = hz;
        }
        exc = a[P - 1].exz;   // read only when plane kb + P is this thread's
        eyc = a[P - 1].eyz;
    }
}

// H of the shell: one thread per column of a shell box (see shell_cell).
template <typename T>
__global__ void __launch_bounds__(kBX * kBY, sizeof(T) == 8 ? 2 : FDTD_SHELL_MINB) shell_h_kernel(const KParams<T> p, const ShellBoxes s)
{
    pdl_wait();
    pdl_trigger();
    ShellCol cl;
    if (shell_cell(s, cl)) h_column<T, false>(p, cl.x, cl.y, cl.k0, cl.k1, read_step<T>(p.ctl));
}

// E^{n+1} of the cells of one column (x, y), planes [k0, k1), that lie outside the working box, from
// H^{n+1/2} of the whole grid (after every H update of the step); loads first within a batch, like
// h_column, with H_x, H_y of the plane below a batch carried over.  Returns the largest |E| sum seen
// on a checked step (0 otherwise).
template <typename T, bool CG>
__device__ __forceinline__ T e_column(const KParams<T>& p, int x, int y, int k0, int k1, int n)
{
    constexpr int P = kShellPZ;
    T emax = T(0);
    {
        const T hinc_n = p.tfsf_i0 >= 0 ? __ldg(p.hinc + n) : T(0);
        const bool check = (n & 15) == 0 || n + 1 == p.n_steps;
        const bool tf = x == p.tfsf_i0;   // H_y(i0-1/2) is scattered field
        const int sx = slab_index(x, p.cpl[0], p.cph[0], p.nx), sy = slab_index(y, p.cpl[1], p.cph[1], p.ny);
        const unsigned nx = (unsigned)p.nx, plane = (unsigned)p.plane, col = (unsigned)y * nx + (unsigned)x;
        const PsiCol pc = psi_col(p, x, y, sx, sy);
        const bool in_dxy = x >= p.db[0] && x < p.db[1] && y >= p.db[2] && y < p.db[3];
        const T* __restrict__ H0 = p.Hn[0];
        const T* __restrict__ H1 = p.Hn[1];
        const T* __restrict__ H2 = p.Hn[2];
        T hxb = T(0), hyb = T(0);   // H_x, H_y of the plane below the batch
        if (k0 > 0) {
            hxb = ldf<CG>(H0 + (unsigned)(k0 - 1) * plane + col);
            hyb = ldf<CG>(H1 + (unsigned)(k0 - 1) * plane + col);
        }
        for (int kb = k0; kb < k1; kb += P) {   // (a compile-time trip bound here costs registers)
            T h[P][3], hm[P][4], e0[P][3], ps[P][6];
            bool on[P];
            int sz[P];
#pragma unroll
            for (int r = 0; r < P; ++r) {
                const int k = kb + r;
                sz[r] = slab_index(k, p.cpl[2], p.cph[2], p.nz);
                on[r] = k < k1 && !(in_dxy && k >= p.db[4] && k < p.db[5]);
                if (k >= k1) continue;
                const unsigned id = (unsigned)k * plane + col;
                h[r][0] = ldf<CG>(H0 + id);
                h[r][1] = ldf<CG>(H1 + id);
                h[r][2] = ldf<CG>(H2 + id);
                hm[r][0] = y > 0 ? ldf<CG>(H2 + id - nx) : T(0);   // H_z(y-1)
                hm[r][1] = y > 0 ? ldf<CG>(H0 + id - nx) : T(0);   // H_x(y-1)
                hm[r][2] = x > 0 ? ldf<CG>(H2 + id - 1) : T(0);    // H_z(x-1)
                hm[r][3] = x > 0 ? ldf<CG>(H1 + id - 1) : T(0);    // H_y(x-1)
                e0[r][0] = ldf<CG>(p.E[0] + id);
                e0[r][1] = ldf<CG>(p.E[1] + id);
                e0[r][2] = ldf<CG>(p.E[2] + id);
                psi_load<T, CG>(p.psiE, pc, (unsigned)k, plane, col, sx, sy, sz[r], ps[r]);
            }
#pragma unroll
            for (int r = 0; r < P; ++r) {
                const int k = kb + r;
                const T hxz = r == 0 ? hxb : h[r - 1][0], hyz = r == 0 ? hyb : h[r - 1][1];
                if (!on[r]) continue;
                const unsigned id = (unsigned)k * plane + col;
                const T rxa = h[r][2] - hm[r][0], rxb = h[r][1] - hyz;
                const T rya = h[r][0] - hxz, ryb = h[r][2] - hm[r][2];
                const T rza = h[r][1] - hm[r][3], rzb = h[r][0] - hm[r][1];
                const bool src = p.nb > 0 && in_box(p.sb, x, y, k);
                T ex, ey, ez;
                if (sx < 0 && sy < 0 && sz[r] < 0 && !src && x > 0 && y > 0 && k > 0) {
                    ex = p.bg_ca[0] * e0[r][0] + p.bg_cbi[0] * (rxa - rxb);
                    ey = p.bg_ca[1] * e0[r][1] + p.bg_cbi[1] * (rya - ryb);
                    ez = p.bg_ca[2] * e0[r][2] + p.bg_cbi[2] * ((tf ? rza - hinc_n : rza) - rzb);
                } else {
                    const T idx = p.inv_dx;
                    T xa = rxa * idx, xb = rxb * idx, ya = rya * idx, yb = ryb * idx, za = rza * idx, zb = rzb * idx;
                    if (tf) za -= hinc_n * idx;
                    if (sy >= 0) {
                        xa = stretch_v(xa, p.pmlE[1], sy, ps[r][0]);
                        zb = stretch_v(zb, p.pmlE[1], sy, ps[r][1]);
                    }
                    if (sz[r] >= 0) {
                        xb = stretch_v(xb, p.pmlE[2], sz[r], ps[r][2]);
                        ya = stretch_v(ya, p.pmlE[2], sz[r], ps[r][3]);
                    }
                    if (sx >= 0) {
                        yb = stretch_v(yb, p.pmlE[0], sx, ps[r][4]);
                        za = stretch_v(za, p.pmlE[0], sx, ps[r][5]);
                    }
                    psi_store(p.psiE, pc, (unsigned)k, plane, col, sx, sy, sz[r], ps[r]);
                    T dxv = xa - xb, dyv = ya - yb, dzv = za - zb;
                    if (src) {
                        dxv += point_drive(p, x, y, k, 0, n);
                        dyv += point_drive(p, x, y, k, 1, n);
                        dzv += point_drive(p, x, y, k, 2, n);
                    }
                    ex = p.bg_ca[0] * e0[r][0] + p.bg_cb[0] * dxv;
                    ey = p.bg_ca[1] * e0[r][1] + p.bg_cb[1] * dyv;
                    ez = p.bg_ca[2] * e0[r][2] + p.bg_cb[2] * dzv;
                    const bool im = x > 0, jm = y > 0, km = k > 0;
                    if (!(jm && km)) ex = e0[r][0];   // PEC walls: components tangential to a wall at index 0 stay zero
                    if (!(km && im)) ey = e0[r][1];
                    if (!(im && jm)) ez = e0[r][2];
                }
                p.En[0][id] = ex;
                p.En[1][id] = ey;
                p.En[2][id] = ez;
                if (check) emax = fmax(emax, fabs(ex) + fabs(ey) + fabs(ez));
            }
            hxb = h[P - 1][0];   // read only when plane kb + P is this thread's
            hyb = h[P - 1][1];
        }
    }
    return emax;
}

// E of the shell cells outside the design box.  It may run concurrently with the design-E kernel: the
// last block of the two launches advances the step.
template <typename T>
__global__ void __launch_bounds__(kBX * kBY, sizeof(T) == 8 ? 2 : FDTD_SHELL_MINB) shell_e_kernel(const KParams<T> p, const ShellBoxes s)
{
    pdl_wait();
    pdl_trigger();
    ShellCol cl;
    const bool live = shell_cell(s, cl);
    const int n = read_step<T>(p.ctl);
    if (live) {
        const T emax = e_column<T, false>(p, cl.x, cl.y, cl.k0, cl.k1, n);
        if (!(emax < p.blowup)) atomicOr(p.ctl + 2, 1);
    }
    finish_step(p.ctl, p.nblocks_e, n);
}

}  // namespace fdtd
