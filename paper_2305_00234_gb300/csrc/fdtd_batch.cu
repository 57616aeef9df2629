// Persistent kernel that advances several independent runs (gradient evaluations of different
// grids, forward or adjoint) together, for serving many small requests at once.
//
// A run's time step is two phases, H then E (the same per-cell updates as the shell kernels and the
// design-E kernel: Eqs. (Maxwells)a-c with CFS-CPML, the blended CCPR update of Eqs. (eps_mixed),
// (sigma_mixed), (Poles_mixed) and the pole recursion), split into work items of sz z planes by cw (x, y)
// columns (per run, by grid size).  The blocks of one launch (a few per SM, persistent) take items from a
// global ticket counter; the items of a launch are numbered round by round (round g = phase g of every
// run still stepping in this launch), so an item only ever waits for items with smaller numbers, which
// blocks that are already running hold: the launch cannot deadlock, and no block needs to be resident
// before another starts.  Per run and slab a counter records completed items; an item of phase q
// (counted from the run's first step) on slab s starts when the slab, and the one slab its stencil
// reaches (s + 1 for H, which reads E of the plane above; s - 1 for E, which reads H of the plane below),
// have completed all q earlier phases.  Write-after-read hazards of the double-buffered fields follow
// from these chains.  E items at the end of a 16-step block fold their voxels' E snapshots into the FP64
// DFT (the voxels an item owns are only ever written by the items of the same slab and chunk).
//
// Every wait is bounded: after wait_ns without progress (or when another block has given up) the
// block records the failure in err and returns; the others see err at their next item and return.
#include "fdtd_kernels.cuh"
#include "fdtd_launch.h"
#include "fdtd_step.cuh"

// Build knobs: FDTD_BATCH_CG 1 loads state through L2 only; 0 (default, measured faster) uses L1-cached
// loads, which the memory model makes safe here: an item's reads follow, through thread 0's ld.acquire.gpu
// of the producers' counters and the block barrier after it, the producers' release (stores, barrier,
// fence, counter increment), so they cannot return lines cached before those stores.
// FDTD_BATCH_INLINE 1 (default, measured faster) inlines the per-column H and E work into the persistent
// loop; 0 compiles them as separate functions.
#ifndef FDTD_BATCH_CG
#define FDTD_BATCH_CG 0
#endif
#ifndef FDTD_BATCH_INLINE
#define FDTD_BATCH_INLINE 1
#endif
#if FDTD_BATCH_INLINE
#define FDTD_BATCH_FN __forceinline__
#else
#define FDTD_BATCH_FN __noinline__
#endif

namespace fdtd {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_acquire_s32(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until *p >= need (or, with flag, *p != 0); false after wait_ns, 2^24 polls, or once err is set.
__device__ __forceinline__ bool wait_count(const unsigned* p, unsigned need, const BatchLaunch& L)
{
    if (ld_acquire_u32(p) >= need) return true;
    const unsigned long long t0 = global_ns();
    for (int it = 0; it < (1 << 24); ++it) {
        __nanosleep(it < 16 ? 32 : 256);
        if (ld_acquire_u32(p) >= need) return true;
        if (ld_acquire_s32(L.err) != 0 || global_ns() - t0 > L.wait_ns) return false;
    }
    return false;
}

// DFT fold of one voxel over steps n0 .. n0 + cnt - 1 (the arithmetic of dft_voxel, the same sums in
// the same order) one component and frequency at a time, which keeps few values live: snapshots are
// re-read from L2 per frequency instead of being held in registers.
template <typename T>
__device__ __forceinline__ void dft_voxel_lean(const DParams<T>& d, long long v, int n0, int cnt)
{
    for (int c = 0; c < 3; ++c) {
        const T* sp = d.snap + (long long)c * d.nd + v;
        for (int f = 0; f < d.nf; ++f) {
            T re = T(0), im = T(0);
            for (int s = 0; s < cnt; ++s) {
                const T e = __ldcg(sp + (long long)((n0 + s) % d.K) * 3 * d.nd);
                const auto ph = __ldg(d.ph + (long long)(n0 + s + 1) * d.nf + f);
                re = fma(e, ph.x, re);
                im = fma(-e, ph.y, im);
            }
            double2* acc = d.dft + (long long)(f * 3 + c) * d.nd + v;
            double2 a = __ldcg(acc);
            a.x += (double)re;
            a.y += (double)im;
            *acc = a;
        }
    }
}

// E of one column of a work item: the cells outside the working box (background, CPML, sources), then
// the three components' samples inside it, then, at the end of a 16-step block, the DFT fold of the
// column's working-box voxels.  Returns the largest |E| seen (for the blow-up test).
template <typename T, int MP>
__device__ __forceinline__ T batch_e_column(const KParams<T>& p, const DParams<T>& dp, const PoleTable<T>& tab, int x,
                                            int y, int k0, int k1, int n)
{
    T em = e_column<T, FDTD_BATCH_CG>(p, x, y, k0, k1, n);
    if (x < p.db[0] || x >= p.db[1] || y < p.db[2] || y >= p.db[3]) return em;
    const int d0 = max(k0, p.db[4]), d1 = min(k1, p.db[5]);
    if (d0 >= d1) return em;
    em = fmax(em, e_design_column<T, MP, 0, FDTD_BATCH_CG>(p, tab, x, y, d0, d1, n));
    em = fmax(em, e_design_column<T, MP, 1, FDTD_BATCH_CG>(p, tab, x, y, d0, d1, n));
    em = fmax(em, e_design_column<T, MP, 2, FDTD_BATCH_CG>(p, tab, x, y, d0, d1, n));
    if ((n - p.snap0 + 1) % p.K == 0 || n + 1 == p.n_steps) {
        const int cnt = (n - p.snap0) % p.K + 1;
        const long long dcol = (long long)(y - p.db[2]) * p.dnx + (x - p.db[0]);
        for (int k = d0; k < d1; ++k) dft_voxel_lean<T>(dp, (long long)(k - p.db[4]) * p.dplane + dcol, n - cnt + 1, cnt);
    }
    return em;
}

// The per-column work of an item, compiled as separate functions so that each is register-allocated on
// its own (inlined into the persistent loop, the H and E paths together would spill).
template <typename T>
__device__ FDTD_BATCH_FN void batch_h(const KParams<T>& p, int x, int y, int k0, int k1, int n)
{
    h_column<T, FDTD_BATCH_CG>(p, x, y, k0, k1, n);
}

template <typename T, int MP>
__device__ FDTD_BATCH_FN T batch_e(const KParams<T>& p, const DParams<T>& dp, const PoleTable<T>& tab, int x, int y,
                                  int k0, int k1, int n)
{
    return batch_e_column<T, MP>(p, dp, tab, x, y, k0, k1, n);
}

// Copy of a plain struct from global to shared memory by the whole block (4-byte words).
template <typename S>
__device__ __forceinline__ void block_copy(S* dst, const S* src)
{
    static_assert(sizeof(S) % 4 == 0, "word copy");
    const unsigned* a = reinterpret_cast<const unsigned*>(src);
    unsigned* b = reinterpret_cast<unsigned*>(dst);
    for (unsigned q = threadIdx.x; q < sizeof(S) / 4; q += blockDim.x) b[q] = __ldcg(a + q);
}

template <typename T, int MP>
__global__ void __launch_bounds__(kBatchThreads, FDTD_BATCH_MINB) batch_kernel(const __grid_constant__ BatchLaunch L)
{
    __shared__ long long s_t;
    __shared__ int s_ok;
    // the item's run parameters, pole table and DFT parameters, in shared memory: the state stores of
    // an item cannot alias them, so they stay cheap to read throughout the item
    __shared__ KParams<T> sp;
    __shared__ DParams<T> sd;
    __shared__ PoleTable<T> stab;
    BatchSlot<T>* slots = (BatchSlot<T>*)L.slots;
    const long long total = L.seg_t0[L.nseg];
    long long next = -1;                // thread 0: ticket taken ahead during the previous item
    for (;;) {
        if (threadIdx.x == 0) {
            long long t = next >= 0 ? next : (long long)atomicAdd(L.ticket, 1ull);
            if (t >= total || ld_acquire_s32(L.err) != 0) t = -1;
            s_t = t;
        }
        __syncthreads();
        const long long t = s_t;
        if (t < 0) return;
        // ticket -> (run, round, slab, chunk)
        int q = 0;
        while (q + 1 < L.nseg && t >= L.seg_t0[q + 1]) ++q;
        const int m = L.seg_m[q];
        const long long per_round = L.pre[m];
        const long long off = t - L.seg_t0[q];
        const long long gr = off / per_round;
        const int g = L.seg_g0[q] + (int)gr;
        const long long u = off - gr * per_round;
        int j = 0;
        while (j + 1 < m && u >= L.pre[j + 1]) ++j;
        BatchSlot<T>& sl = slots[L.slot[j]];
        const int w = (int)(u - L.pre[j]);
        const int s = w / sl.nxyc, c = w - s * sl.nxyc;
        const int n = sl.n0 + (g >> 1), kind = g & 1;     // kind 0: H phase of step n, 1: E phase
        const unsigned need = (unsigned)(2 * n + kind) * (unsigned)sl.nxyc;
        block_copy(&sp, &sl.kp[n & 1]);
        if (kind == 1) {
            block_copy(&sd, &sl.dp);
            block_copy(&stab, sl.kp[0].poles);
        }
        if (threadIdx.x == 0) {
            bool ok = wait_count(sl.prog + s, need, L);
            if (ok && kind == 0 && s + 1 < sl.nslab) ok = wait_count(sl.prog + s + 1, need, L);
            if (ok && kind == 1 && s > 0) ok = wait_count(sl.prog + s - 1, need, L);
            if (ok && L.gate && t == 0) ok = wait_count((const unsigned*)L.gate, 1u, L);   // test hook
            if (!ok && atomicCAS(L.err, 0, 1) == 0) atomicExch(L.err + 1, (int)t);
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return;
        // the next ticket, taken now so that its round trip overlaps this item's work (an item only
        // waits for smaller tickets, so holding two cannot deadlock)
        if (threadIdx.x == 0) next = (long long)atomicAdd(L.ticket, 1ull);
        const KParams<T>& p = sp;
        const int nx = p.nx, nxy = p.nx * p.ny;
        const int k0 = s * sl.sz, k1 = min(k0 + sl.sz, p.nz);
        const int ce = min((c + 1) * sl.cw, nxy);
        T emax = T(0);
        for (int col = c * sl.cw + (int)threadIdx.x; col < ce; col += kBatchThreads) {
            const int y = col / nx, x = col - y * nx;
            if (kind == 0)
                batch_h<T>(p, x, y, k0, k1, n);
            else
                emax = fmax(emax, batch_e<T, MP>(p, sd, stab, x, y, k0, k1, n));
        }
        if (kind == 1 && !(emax < p.blowup)) atomicOr(p.ctl + 2, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(sl.prog + s, 1u);
        }
    }
}

template <typename T>
const void* batch_kernel_fn(int bucket)
{
    switch (bucket) {
    case 0:
    case 4: return (const void*)batch_kernel<T, 4>;
    case 8: return (const void*)batch_kernel<T, 8>;
    default: return (const void*)batch_kernel<T, 16>;
    }
}

template <typename T>
cudaError_t batch_blocks_per_sm(int bucket, int* out)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, batch_kernel_fn<T>(bucket), kBatchThreads, 0);
}

template const void* batch_kernel_fn<float>(int);
template cudaError_t batch_blocks_per_sm<float>(int, int*);

}  // namespace fdtd
