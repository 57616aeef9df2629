// Launch wrappers and helper kernels; explicit FP32 / FP64 instantiations.
#include <utility>

#include "fdtd_design2.cuh"
#include "fdtd_kernels.cuh"
#include "fdtd_launch.h"
#include "fdtd_shell2.cuh"
#include "fdtd_step.cuh"

namespace fdtd {

__global__ void gap_gather_kernel(const double2* dft, long long nd, int nf, int d0, int d2, int d4, int dnx, int dny,
                                  int g0, int g1, int g2, int g3, int g4, int g5, double2* out)
{
    const int gnx = g1 - g0, gny = g3 - g2, gnz = g5 - g4;
    const long long ng = (long long)gnx * gny * gnz;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ng * 3 * nf) return;
    const long long gv = t % ng;
    const long long fc = t / ng;
    const int i = g0 + (int)(gv % gnx), j = g2 + (int)((gv / gnx) % gny), k = g4 + (int)(gv / ((long long)gnx * gny));
    const long long dv = ((long long)(k - d4) * dny + (j - d2)) * dnx + (i - d0);
    out[t] = dft[fc * nd + dv];
}

// Density import: float / double source -> T, with a range / finiteness check (flag bit 1).
template <typename T, typename S>
__global__ void rho_import_kernel(const S* src, long long n, T* dst, int* flag)
{
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const S r = src[v];
    if (!(r >= S(0) && r <= S(1))) atomicOr(flag, 2);
    dst[v] = (T)r;
}

template <typename T>
__global__ void to_double_kernel(const T* src, long long n, double* dst)
{
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) dst[v] = (double)src[v];
}

// Integer maps from the same index helpers the update kernels use.
template <typename T>
__global__ void index_map_kernel(const KParams<T> p, int which, int32_t* out)
{
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= p.nx || j >= p.ny) return;
    const long long id = ((long long)k * p.ny + j) * p.nx + i;
    const bool in_d = in_box(p.db, i, j, k);
    const bool in_g = in_d && in_box(p.gb, i, j, k);
    if (which == 2) {
        out[id] = in_d ? (int32_t)(((long long)(k - p.db[4]) * p.dny + (j - p.db[2])) * p.dnx + (i - p.db[0])) : -1;
        return;
    }
    if (which == 3) {
        out[id] = in_g ? (int32_t)(((long long)(k - p.gb[4]) * p.gny + (j - p.gb[2])) * p.gnx + (i - p.gb[0])) : -1;
        return;
    }
    const int l[3] = {i, j, k};
    const int sl[3] = {slab_index(i, p.cpl[0], p.cph[0], p.nx), slab_index(j, p.cpl[1], p.cph[1], p.ny),
                       slab_index(k, p.cpl[2], p.cph[2], p.nz)};
    for (int c = 0; c < 3; ++c) {
        int32_t v = 0;
        for (int t = 0; t < 2; ++t) {
            const int a = (c + 1 + t) % 3;
            const T* tab = (which == 0) ? p.pmlE[a] : p.pmlH[a];
            if (sl[a] >= 0 && tab[4 * sl[a] + 2] != T(0)) v |= 1 << (3 + t);
        }
        if (which == 0) {
            v |= in_g ? 2 : ((in_d && in_box(p.mb[c], i, j, k)) ? 1 : 0);
            bool fixed = false;
            for (int a = 0; a < 3; ++a)
                if (a != c && l[a] == 0) fixed = true;
            if (fixed) v |= 4;
            if (p.nb > 0 && in_box(p.sb, i, j, k)) {
                const long long lv = ((long long)(k - p.sb[4]) * (p.sb[3] - p.sb[2]) + (j - p.sb[2])) * (p.sb[1] - p.sb[0]) + (i - p.sb[0]);
                if (p.src_r[(lv * 3 + c) * p.nb] != T(0)) v |= 32;
            }
        }
        out[(long long)c * p.ncell + id] = v;
    }
}

static dim3 grid3(int nx, int ny, int nz) { return dim3((nx + kBX - 1) / kBX, (ny + kBY - 1) / kBY, nz); }

// Launch of a kernel of the step chain; pdl: as a programmatic dependent launch (its blocks may start
// before the kernel before it in the stream has completed; see pdl_wait / pdl_trigger).
template <typename... KArgs, typename... Args>
static cudaError_t launch_chain(void (*k)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t s, bool pdl,
                                Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

int pole_bucket(int max_poles)
{
    return max_poles == 0 ? 0 : max_poles <= 4 ? 4 : max_poles <= 8 ? 8 : 16;
}

template <typename T>
cudaError_t prepare_step()
{
    return cudaFuncSetAttribute(step_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)StepSmem<T>::total);
}

// A kernel node of a step graph (no dependencies yet; the host adds them).
template <typename... KArgs, typename... Args>
static cudaError_t graph_kernel(cudaGraph_t g, cudaGraphNode_t* node, void (*k)(KArgs...), dim3 grid, dim3 block,
                                size_t smem, Args... args)
{
    void* ptrs[] = {(void*)&args...};
    cudaKernelNodeParams kp = {};
    kp.func = (void*)k;
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = ptrs;
    return cudaGraphAddKernelNode(node, g, nullptr, 0, &kp);
}

template <typename T>
cudaError_t graph_step(cudaGraph_t g, cudaGraphNode_t* node, const KParams<T>& p, const StepMaps& m)
{
    const dim3 grid((p.ib[1] - p.ib[0] + kTX - 1) / kTX, (p.ib[3] - p.ib[2] + kTY - 1) / kTY, (p.ib[5] - p.ib[4] + p.kc - 1) / p.kc);
    return graph_kernel(g, node, step_kernel<T>, grid, dim3(kPX, kTY), StepSmem<T>::total, p, m);
}

template <typename T>
cudaError_t graph_shell(cudaGraph_t g, cudaGraphNode_t* node, const KParams<T>& p, const ShellBoxes& s, bool e_part)
{
    const dim3 grid(s.first[s.n]), b(kBX, kBY);
    if constexpr (sizeof(T) == 4) {
        if (s.pair)
            return e_part ? graph_kernel(g, node, shell_e2_kernel, grid, b, 0, p, s)
                          : graph_kernel(g, node, shell_h2_kernel, grid, b, 0, p, s);
    }
    return e_part ? graph_kernel(g, node, shell_e_kernel<T>, grid, b, 0, p, s)
                  : graph_kernel(g, node, shell_h_kernel<T>, grid, b, 0, p, s);
}

// Grid of the design-E kernel: one block per (p.edz planes, component) of 32 x 8 columns (32 x 8 column
// pairs for the paired kernel).
template <typename T>
static dim3 design_grid(const KParams<T>& p)
{
    const dim3 g3 = grid3((p.db[1] - p.db[0]) / (p.ed_pair ? 2 : 1), p.db[3] - p.db[2], p.db[5] - p.db[4]);
    const unsigned nxy = (unsigned)(p.db[1] - p.db[0]) * (unsigned)(p.db[3] - p.db[2]);
    if (FDTD_ED_FLAT && !p.ed_pair)
        return dim3((nxy + kBX * kBY - 1) / (kBX * kBY), 1, 3 * ((g3.z + p.edz - 1) / p.edz));
    return dim3(g3.x, g3.y, 3 * ((g3.z + p.edz - 1) / p.edz));
}

template <typename T>
cudaError_t graph_e_design(cudaGraph_t g, cudaGraphNode_t* node, const KParams<T>& p, const PoleTable<T>& tab, int bucket)
{
    const dim3 b(kBX, kBY), grid = design_grid(p);
    if constexpr (sizeof(T) == 4) {
        if (p.ed_pair) switch (bucket) {
            case 0: return graph_kernel(g, node, e_design2_kernel<0>, grid, b, 0, p, tab);
            case 4: return graph_kernel(g, node, e_design2_kernel<4>, grid, b, 0, p, tab);
            case 8: return graph_kernel(g, node, e_design2_kernel<8>, grid, b, 0, p, tab);
            default: return cudaErrorInvalidValue;   // the host pairs only up to 8 poles a component
            }
    }
    switch (bucket) {
    case 0: return graph_kernel(g, node, e_design_kernel<T, 0>, grid, b, 0, p, tab);
    case 4: return graph_kernel(g, node, e_design_kernel<T, 4>, grid, b, 0, p, tab);
    case 8: return graph_kernel(g, node, e_design_kernel<T, 8>, grid, b, 0, p, tab);
    default: return graph_kernel(g, node, e_design_kernel<T, 16>, grid, b, 0, p, tab);
    }
}

template <typename T>
cudaError_t graph_dft(cudaGraph_t g, cudaGraphNode_t* node, const DParams<T>& d, int cnt)
{
    return graph_kernel(g, node, dft_kernel<T>, dim3((unsigned)((d.nd + kReduceThreads - 1) / kReduceThreads)),
                        dim3(kReduceThreads), 0, d, cnt);
}

template <typename T>
unsigned step_blocks(const KParams<T>& p)
{
    return (unsigned)((p.ib[1] - p.ib[0] + kTX - 1) / kTX) * (unsigned)((p.ib[3] - p.ib[2] + kTY - 1) / kTY) *
           (unsigned)((p.ib[5] - p.ib[4] + p.kc - 1) / p.kc);
}

template <typename T>
cudaError_t launch_step(const KParams<T>& p, const StepMaps& m, cudaStream_t s, bool pdl)
{
    const dim3 g((p.ib[1] - p.ib[0] + kTX - 1) / kTX, (p.ib[3] - p.ib[2] + kTY - 1) / kTY, (p.ib[5] - p.ib[4] + p.kc - 1) / p.kc);
    return launch_chain(step_kernel<T>, g, dim3(kPX, kTY), StepSmem<T>::total, s, pdl, p, m);
}

// Launches with fewer blocks than this (two per SM) get shorter per-thread columns, so that small
// grids still spread over the SMs; above it long columns win (measured on 256^3 and 96x170x170).
constexpr unsigned kMinColumnBlocks = 2 * 152;

// Columns of kShellKZ planes, shortened (by kShellPZ at a time) while the launch has fewer than
// FDTD_SHELL_MINCOLS blocks.
#ifndef FDTD_SHELL_MINCOLS
#define FDTD_SHELL_MINCOLS kMinColumnBlocks
#endif
unsigned shell_blocks(ShellBoxes& s)
{
    unsigned t = 0;
    for (s.kz = kShellKZ;; s.kz -= kShellPZ) {
        t = 0;
        for (int q = 0; q < s.n; ++q) {
            const int* B = s.b[q];
            s.first[q] = t;
            const unsigned wxy = (unsigned)(B[1] - B[0]) / (s.pair ? 2u : 1u) * (unsigned)(B[3] - B[2]);
            t += (wxy + kShellCells - 1) / kShellCells * (unsigned)((B[5] - B[4] + s.kz - 1) / s.kz);
        }
        s.first[s.n] = t;
        if (t >= FDTD_SHELL_MINCOLS || s.kz <= kShellPZ) break;
    }
    return t;
}

template <typename T>
cudaError_t launch_shell(const KParams<T>& p, const ShellBoxes& s, bool e_part, cudaStream_t st, bool pdl)
{
    const unsigned nb = s.first[s.n];
    if (nb == 0) return cudaSuccess;
    const dim3 b(kBX, kBY);
    if constexpr (sizeof(T) == 4) {
        if (s.pair)
            return e_part ? launch_chain(shell_e2_kernel, dim3(nb), b, 0, st, pdl, p, s)
                          : launch_chain(shell_h2_kernel, dim3(nb), b, 0, st, pdl, p, s);
    }
    return e_part ? launch_chain(shell_e_kernel<T>, dim3(nb), b, 0, st, pdl, p, s)
                  : launch_chain(shell_h_kernel<T>, dim3(nb), b, 0, st, pdl, p, s);
}

template <typename T>
cudaError_t launch_e_design(const KParams<T>& p, const PoleTable<T>& tab, int bucket, cudaStream_t s, bool pdl)
{
    if (p.nd == 0) return cudaSuccess;
    const dim3 b(kBX, kBY), g = design_grid(p);
    if constexpr (sizeof(T) == 4) {
        if (p.ed_pair) switch (bucket) {
            case 0: return launch_chain(e_design2_kernel<0>, g, b, 0, s, pdl, p, tab);
            case 4: return launch_chain(e_design2_kernel<4>, g, b, 0, s, pdl, p, tab);
            case 8: return launch_chain(e_design2_kernel<8>, g, b, 0, s, pdl, p, tab);
            default: return cudaErrorInvalidValue;   // the host pairs only up to 8 poles a component
            }
    }
    switch (bucket) {
    case 0: return launch_chain(e_design_kernel<T, 0>, g, b, 0, s, pdl, p, tab);
    case 4: return launch_chain(e_design_kernel<T, 4>, g, b, 0, s, pdl, p, tab);
    case 8: return launch_chain(e_design_kernel<T, 8>, g, b, 0, s, pdl, p, tab);
    default: return launch_chain(e_design_kernel<T, 16>, g, b, 0, s, pdl, p, tab);
    }
}

template <typename T>
cudaError_t launch_dft(const DParams<T>& d, int cnt, cudaStream_t s, bool pdl)
{
    if (d.nd == 0 || cnt <= 0) return cudaSuccess;
    return launch_chain(dft_kernel<T>, dim3((unsigned)((d.nd + kReduceThreads - 1) / kReduceThreads)),
                        dim3(kReduceThreads), 0, s, pdl, d, cnt);
}


// Columns of kEdZ planes, halved while the launch has fewer than FDTD_ED_MINCOLS blocks (default: one
// wave of five resident blocks per SM; measured 3.7% faster than two blocks per SM on the 96 x 170 x 170
// paper grid, whose design box is 26 cells deep in x).
#ifndef FDTD_ED_MINCOLS
#define FDTD_ED_MINCOLS (5 * 152)
#endif
unsigned design_blocks(int dnx, int dny, int dnz, int& edz, bool flat)
{
    const dim3 g = grid3(dnx, dny, dnz);
    const unsigned gxy = flat ? ((unsigned)dnx * (unsigned)dny + kBX * kBY - 1) / (kBX * kBY) : g.x * g.y;
    unsigned t = 0;
    for (edz = kEdZ;; edz = (edz + 1) / 2) {
        t = gxy * 3 * ((g.z + edz - 1) / edz);
        if (t >= FDTD_ED_MINCOLS || edz == 1) break;
    }
    return t;
}

template <typename T>
cudaError_t launch_grad(const GParams<T>& g, unsigned nblocks, cudaStream_t s)
{
    grad_kernel<T><<<nblocks, kReduceThreads, 0, s>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_gap_gather(const double2* dft, long long nd, int nf, const int* db, int dnx, int dny, const int* gb,
                              double2* out, cudaStream_t s)
{
    const long long ng = (long long)(gb[1] - gb[0]) * (gb[3] - gb[2]) * (gb[5] - gb[4]);
    const long long nt = ng * 3 * nf;
    if (nt == 0) return cudaSuccess;
    gap_gather_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(dft, nd, nf, db[0], db[2], db[4], dnx, dny, gb[0], gb[1],
                                                                   gb[2], gb[3], gb[4], gb[5], out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rho_import(const void* src, int dtype, long long n, T* dst, int* flag, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (dtype == 0)
        rho_import_kernel<T, float><<<nb, 256, 0, s>>>((const float*)src, n, dst, flag);
    else
        rho_import_kernel<T, double><<<nb, 256, 0, s>>>((const double*)src, n, dst, flag);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_to_double(const T* src, long long n, double* dst, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    to_double_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, n, dst);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_index_map(const KParams<T>& p, int which, int32_t* out, cudaStream_t s)
{
    index_map_kernel<T><<<grid3(p.nx, p.ny, p.nz), dim3(kBX, kBY), 0, s>>>(p, which, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_design_e(const KParams<T>& p, T* out, cudaStream_t s)
{
    if (p.nd == 0) return cudaSuccess;
    gather_design_e_kernel<T><<<(unsigned)((p.nd + 255) / 256), 256, 0, s>>>(p, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_paper_drive(const T* gh, T* drive, int M, int ns, double eps0, cudaStream_t s)
{
    const long long n = (long long)M * ns;
    if (n == 0) return cudaSuccess;
    paper_drive_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(gh, drive, M, ns, eps0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_paper_grad(const PParams<T>& g, cudaStream_t s)
{
    if (g.nd == 0) return cudaSuccess;
    paper_grad_kernel<T><<<(unsigned)((g.nd + 255) / 256), 256, 0, s>>>(g);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rho_scatter(const void* src, int dtype, long long n, const long long off[4], const int md[3][3],
                               int dnx, int dny, long long nd, T* dst, int* flag, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int3 m0 = make_int3(md[0][0], md[0][1], md[0][2]), m1 = make_int3(md[1][0], md[1][1], md[1][2]);
    const int3 m2 = make_int3(md[2][0], md[2][1], md[2][2]);
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (dtype == 0)
        rho_scatter_kernel<T, float><<<nb, 256, 0, s>>>((const float*)src, n, off[1], off[2], m0, m1, m2, dnx, dny, nd, dst, flag);
    else
        rho_scatter_kernel<T, double><<<nb, 256, 0, s>>>((const double*)src, n, off[1], off[2], m0, m1, m2, dnx, dny, nd, dst, flag);
    return cudaGetLastError();
}

#define FDTD_INSTANTIATE(T)                                                                              \
    template cudaError_t prepare_step<T>();                                                              \
    template unsigned step_blocks<T>(const KParams<T>&);                                                \
    template cudaError_t graph_step<T>(cudaGraph_t, cudaGraphNode_t*, const KParams<T>&, const StepMaps&); \
    template cudaError_t graph_shell<T>(cudaGraph_t, cudaGraphNode_t*, const KParams<T>&, const ShellBoxes&, bool); \
    template cudaError_t graph_e_design<T>(cudaGraph_t, cudaGraphNode_t*, const KParams<T>&, const PoleTable<T>&, int); \
    template cudaError_t graph_dft<T>(cudaGraph_t, cudaGraphNode_t*, const DParams<T>&, int);           \
    template cudaError_t launch_step<T>(const KParams<T>&, const StepMaps&, cudaStream_t, bool);         \
    template cudaError_t launch_shell<T>(const KParams<T>&, const ShellBoxes&, bool, cudaStream_t, bool); \
    template cudaError_t launch_e_design<T>(const KParams<T>&, const PoleTable<T>&, int, cudaStream_t, bool); \
    template cudaError_t launch_dft<T>(const DParams<T>&, int, cudaStream_t, bool);                      \
    template cudaError_t launch_grad<T>(const GParams<T>&, unsigned, cudaStream_t);                      \
    template cudaError_t launch_rho_import<T>(const void*, int, long long, T*, int*, cudaStream_t);      \
    template cudaError_t launch_rho_scatter<T>(const void*, int, long long, const long long*, const int (*)[3], int, \
                                               int, long long, T*, int*, cudaStream_t);                   \
    template cudaError_t launch_to_double<T>(const T*, long long, double*, cudaStream_t);                \
    template cudaError_t launch_index_map<T>(const KParams<T>&, int, int32_t*, cudaStream_t);            \
    template cudaError_t launch_gather_design_e<T>(const KParams<T>&, T*, cudaStream_t);                  \
    template cudaError_t launch_paper_drive<T>(const T*, T*, int, int, double, cudaStream_t);             \
    template cudaError_t launch_paper_grad<T>(const PParams<T>&, cudaStream_t);

FDTD_INSTANTIATE(float)
FDTD_INSTANTIATE(double)

}  // namespace fdtd
