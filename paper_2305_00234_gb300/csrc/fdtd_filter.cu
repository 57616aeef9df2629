// Density filter, smoothed-Heaviside projection and their chain rule (the paper's Sec. "Filtering and
// projection", Eqs. (FilterFunction), (Projection), (GradientsFiltered)) on the design box.
//
// The cone filter is a 3-D correlation with w(d) = R - |d| over |d| < R (voxels), neighbourhoods cut at
// the box faces.  cone_kernel computes one output voxel per thread for an 8x8x8 tile: the block stages
// the tile plus a halo of n = ceil(R)-1 voxels of input (zero outside the box) and the (2n+1)^3 weight
// table in shared memory, then every thread sums its sphere; the weight read is a broadcast and the
// input reads of a warp are consecutive in x; each row runs over the sphere's taps only.  Two shared-
// memory loads per FMA bound it (about 7100 taps per output at R = 12): 21 ms for the forward + chain
// rule pair on a 128^3 design box, about 1% of one gradient evaluation there.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "fdtd_ccpr.h"
#include "fdtd_kernels.cuh"

namespace fdtd {
void set_thread_error(const std::string& msg);
}

namespace {

constexpr int kT = 8;             // output tile edge
constexpr int kMaxHalo = 11;      // R <= 12
constexpr int kThreads = kT * kT * kT;

// Smallest pitch >= L that is 8 mod 32: a warp reads 4 rows of 8 consecutive floats.
__host__ __device__ inline int row_pitch(int L) { return L + ((8 - L) % 32 + 32) % 32; }

struct ConvArgs {
    const float* in;   // nullptr: the indicator of the box (ones inside)
    float* out;
    const float* div;  // optional: out = sum / div
    float* proj;       // optional: projection of out
    int nx, ny, nz, n;
    float R, beta, eta, pden;
};

__global__ void __launch_bounds__(kThreads) cone_kernel(const ConvArgs a)
{
    extern __shared__ float sm[];
    const int n = a.n, W = 2 * n + 1, L = kT + 2 * n;
    const int P = row_pitch(L);           // x pitch of the tile; the 4 rows of a warp hit distinct banks
    float* wt = sm;                       // W^3 weights
    float* tile = sm + W * W * W;         // L x L x P inputs
    int* span = (int*)(tile + L * L * P); // per (dz, dy) row: first and one-past-last nonzero weight
    const int tid = threadIdx.x;
    for (int q = tid; q < W * W * W; q += kThreads) {
        const int dx = q % W - n, dy = (q / W) % W - n, dz = q / (W * W) - n;
        const float d = sqrtf((float)(dx * dx + dy * dy + dz * dz));
        wt[q] = d < a.R ? a.R - d : 0.f;
    }
    __syncthreads();
    for (int r = tid; r < W * W; r += kThreads) {   // the sphere's extent in each row (zero taps skipped)
        int lo = W, hi = 0;
        for (int dx = 0; dx < W; ++dx)
            if (wt[r * W + dx] != 0.f) {
                lo = min(lo, dx);
                hi = dx + 1;
            }
        span[2 * r] = lo;
        span[2 * r + 1] = hi;
    }
    const int x0 = blockIdx.x * kT - n, y0 = blockIdx.y * kT - n, z0 = blockIdx.z * kT - n;
    for (int q = tid; q < L * L * L; q += kThreads) {
        const int lx = q % L, ly = (q / L) % L, lz = q / (L * L);
        const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
        const bool inside = x >= 0 && x < a.nx && y >= 0 && y < a.ny && z >= 0 && z < a.nz;
        tile[(lz * L + ly) * P + lx] = inside ? (a.in ? a.in[((long long)z * a.ny + y) * a.nx + x] : 1.f) : 0.f;
    }
    __syncthreads();
    const int tx = tid % kT, ty = (tid / kT) % kT, tz = tid / (kT * kT);
    const int x = blockIdx.x * kT + tx, y = blockIdx.y * kT + ty, z = blockIdx.z * kT + tz;
    float s = 0.f;
    for (int dz = 0; dz < W; ++dz)
        for (int dy = 0; dy < W; ++dy) {
            const float* trow = tile + ((tz + dz) * L + (ty + dy)) * P + tx;
            const float* wrow = wt + (dz * W + dy) * W;
            const int lo = span[2 * (dz * W + dy)], hi = span[2 * (dz * W + dy) + 1];
            for (int dx = lo; dx < hi; ++dx) s = fmaf(wrow[dx], trow[dx], s);
        }
    if (x >= a.nx || y >= a.ny || z >= a.nz) return;
    const long long o = ((long long)z * a.ny + y) * a.nx + x;
    if (a.div) s /= a.div[o];
    a.out[o] = s;
    if (a.proj) a.proj[o] = (tanhf(a.beta * a.eta) + tanhf(a.beta * (s - a.eta))) / a.pden;
}

// g = dF/drho_b * drho_b/drho_t / W  (the input of the transposed filter)
__global__ void chain_pre_kernel(const float* dFb, const float* rho_t, const float* Wsum, float* g, long long nv,
                                 float beta, float eta, float pden)
{
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const float t = tanhf(beta * (rho_t[v] - eta));
    g[v] = dFb[v] * beta * (1.f - t * t) / pden / Wsum[v];
}

fdtd_status fail(fdtd_status c, const std::string& m)
{
    fdtd::set_thread_error(m);
    return c;
}

fdtd_status check(int nx, int ny, int nz, double R, double beta, double eta)
{
    if (nx < 1 || ny < 1 || nz < 1) return fail(FDTD_ERR_ARG, "filter: empty box");
    if (!(R > 0.0 && R <= kMaxHalo + 1)) return fail(FDTD_ERR_ARG, "filter: radius must be in (0, 12] voxels");
    if (!(beta > 0.0) || !(eta >= 0.0 && eta <= 1.0)) return fail(FDTD_ERR_ARG, "projection: beta > 0, eta in [0,1]");
    return FDTD_OK;
}

cudaError_t conv(const float* in, float* out, const float* div, float* proj, int nx, int ny, int nz, double R, double beta,
                 double eta, cudaStream_t s)
{
    ConvArgs a;
    a.in = in;
    a.out = out;
    a.div = div;
    a.proj = proj;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.n = (int)std::ceil(R) - 1;
    a.R = (float)R;
    a.beta = (float)beta;
    a.eta = (float)eta;
    a.pden = (float)(std::tanh(beta * eta) + std::tanh(beta * (1.0 - eta)));
    const int W = 2 * a.n + 1, L = kT + 2 * a.n;
    const size_t smem = sizeof(float) * (size_t)(W * W * W + L * L * row_pitch(L)) + sizeof(int) * 2 * (size_t)(W * W);
    cudaError_t e = cudaFuncSetAttribute(cone_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 g((nx + kT - 1) / kT, (ny + kT - 1) / kT, (nz + kT - 1) / kT);
    cone_kernel<<<g, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

extern "C" fdtd_status fdtd_filter_project(const float* rho, float* rho_t, float* rho_b, int nx, int ny, int nz,
                                           double R, double beta, double eta, void* cuda_stream)
{
    if (!rho || !rho_t || !rho_b) return fail(FDTD_ERR_ARG, "filter: null pointer");
    if (fdtd_status st = check(nx, ny, nz, R, beta, eta)) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t nv = (size_t)nx * ny * nz;
    float* Wsum = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&Wsum, nv * sizeof(float), s);
    if (e != cudaSuccess) return fail(FDTD_ERR_OOM, std::string("filter: ") + cudaGetErrorString(e));
    e = conv(nullptr, Wsum, nullptr, nullptr, nx, ny, nz, R, beta, eta, s);                 // normalising sums
    if (e == cudaSuccess) e = conv(rho, rho_t, Wsum, rho_b, nx, ny, nz, R, beta, eta, s);   // filter + project
    cudaFreeAsync(Wsum, s);
    if (e != cudaSuccess) return fail(FDTD_ERR_CUDA, std::string("filter: ") + cudaGetErrorString(e));
    return FDTD_OK;
}

extern "C" fdtd_status fdtd_filter_project_grad(const float* rho_t, const float* dF_drho_b, float* dF_drho, int nx,
                                                int ny, int nz, double R, double beta, double eta, void* cuda_stream)
{
    if (!rho_t || !dF_drho_b || !dF_drho) return fail(FDTD_ERR_ARG, "filter grad: null pointer");
    if (fdtd_status st = check(nx, ny, nz, R, beta, eta)) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t nv = (size_t)nx * ny * nz;
    float* buf = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&buf, 2 * nv * sizeof(float), s);
    if (e != cudaSuccess) return fail(FDTD_ERR_OOM, std::string("filter grad: ") + cudaGetErrorString(e));
    float* Wsum = buf;
    float* g = buf + nv;
    const float pden = (float)(std::tanh(beta * eta) + std::tanh(beta * (1.0 - eta)));
    e = conv(nullptr, Wsum, nullptr, nullptr, nx, ny, nz, R, beta, eta, s);
    if (e == cudaSuccess) {
        chain_pre_kernel<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(dF_drho_b, rho_t, Wsum, g, (long long)nv, (float)beta,
                                                                       (float)eta, pden);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = conv(g, dF_drho, nullptr, nullptr, nx, ny, nz, R, beta, eta, s);   // transposed filter
    cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return fail(FDTD_ERR_CUDA, std::string("filter grad: ") + cudaGetErrorString(e));
    return FDTD_OK;
}
