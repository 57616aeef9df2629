// Density filter, smoothed-Heaviside projection and their chain rule (the paper's Sec. "Filtering and
// projection", Eqs. (FilterFunction), (Projection), (GradientsFiltered)) on the design box.
//
// The cone filter is a 3-D correlation with w(d) = R - |d| over |d| < R (voxels), neighbourhoods cut at
// the box faces.  cone_kernel computes a 32x4x8 output tile per block, four x-adjacent outputs per
// thread: the block stages the tile plus a halo of n = ceil(R)-1 voxels of input (zero outside the box)
// and the sphere's weights, row by row, in shared memory; every thread then runs over the sphere's taps
// with a sliding window of four inputs, so one input load and one (broadcast) weight load feed four
// FMAs.  (Eight outputs per thread with 128-thread blocks measured slower: 3.1 against 2.4 ms per 128^3
// correlation at R = 12.)  The normalising sums (the cone summed over the part of the sphere inside the
// box) depend only on each voxel's distances to the box faces: wsum_kernel takes them from a
// summed-volume table of the weights by inclusion-exclusion.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "fdtd_ccpr.h"
#include "fdtd_kernels.cuh"

namespace fdtd {
void set_thread_error(const std::string& msg);
}

namespace {

// Output tile of one block: 32 x 4 x 8 voxels; a thread owns 4 consecutive x outputs (a warp: 8 such
// groups x 4 rows), so each input it loads from shared memory feeds four FMAs.
constexpr int kGX = 8, kXR = 4, kTY = 4, kTZ = 8;
constexpr int kOX = kGX * kXR;                 // 32 outputs along x
constexpr int kMaxHalo = 11;                   // R <= 12
constexpr int kThreads = kGX * kTY * kTZ;      // 256

// Smallest pitch >= L that is 1 mod 4: the 8 groups (stride 4) x 4 rows of a warp hit 32 banks.
__host__ __device__ inline int row_pitch(int L) { return L + ((1 - L) % 4 + 4) % 4; }

struct ConvArgs {
    const float* in;   // nullptr: the indicator of the box (ones inside)
    float* out;
    const float* div;  // optional: out = sum / div
    float* proj;       // optional: projection of out
    int nx, ny, nz, n, ntaps;
    float R, beta, eta, pden;
};

// Cone weight of offset (dx, dy, dz): R - |d| inside the sphere |d| < R, else 0 (not stored).
__host__ __device__ inline float cone_weight(int dx, int dy, int dz, float R, bool& inside)
{
    const float d = sqrtf((float)(dx * dx + dy * dy + dz * dz));
    inside = d < R;
    return R - d;
}

__global__ void __launch_bounds__(kThreads) cone_kernel(const ConvArgs a)
{
    extern __shared__ float sm[];
    const int n = a.n, W = 2 * n + 1;
    const int Lx = kOX + 2 * n, Ly = kTY + 2 * n, Lz = kTZ + 2 * n, P = row_pitch(Lx);
    float* tile = sm;                                   // Lz x Ly x P inputs
    float* wc = tile + (size_t)Lz * Ly * P;             // the sphere's weights, row by row
    int* rows = (int*)(wc + a.ntaps);                   // per (dz, dy) row: first tap, end, offset in wc
    const int tid = threadIdx.x;
    for (int r = tid; r < W * W; r += kThreads) {
        int lo = W, hi = 0;
        for (int i = 0; i < W; ++i) {
            bool in;
            cone_weight(i - n, r % W - n, r / W - n, a.R, in);
            if (in) {
                lo = min(lo, i);
                hi = i + 1;
            }
        }
        rows[3 * r] = lo;
        rows[3 * r + 1] = hi;
    }
    __syncthreads();
    if (tid == 0) {
        int off = 0;
        for (int r = 0; r < W * W; ++r) {
            rows[3 * r + 2] = off;
            off += max(0, rows[3 * r + 1] - rows[3 * r]);
        }
    }
    __syncthreads();
    for (int r = tid; r < W * W; r += kThreads) {
        bool in;
        for (int i = rows[3 * r]; i < rows[3 * r + 1]; ++i)
            wc[rows[3 * r + 2] + i - rows[3 * r]] = cone_weight(i - n, r % W - n, r / W - n, a.R, in);
    }
    const int x0 = blockIdx.x * kOX - n, y0 = blockIdx.y * kTY - n, z0 = blockIdx.z * kTZ - n;
    for (int q = tid; q < Lx * Ly * Lz; q += kThreads) {
        const int lx = q % Lx, ly = (q / Lx) % Ly, lz = q / (Lx * Ly);
        const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
        const bool inside = x >= 0 && x < a.nx && y >= 0 && y < a.ny && z >= 0 && z < a.nz;
        tile[(lz * Ly + ly) * P + lx] = inside ? (a.in ? a.in[((long long)z * a.ny + y) * a.nx + x] : 1.f) : 0.f;
    }
    __syncthreads();
    const int g = tid % kGX, ty = (tid / kGX) % kTY, tz = tid / (kGX * kTY);
    // per output the taps are summed in the order (dz, dy, dx), one accumulator each; a sliding window
    // of four inputs serves the thread's four x-adjacent outputs
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (int dz = 0; dz < W; ++dz)
        for (int dy = 0; dy < W; ++dy) {
            const int r = dz * W + dy, lo = rows[3 * r], hi = rows[3 * r + 1];
            if (lo >= hi) continue;
            const float* trow = tile + ((tz + dz) * Ly + (ty + dy)) * P + kXR * g;
            const float* wr = wc + rows[3 * r + 2] - lo;
            float v0 = trow[lo], v1 = trow[lo + 1], v2 = trow[lo + 2];
            for (int i = lo; i < hi; ++i) {
                const float v3 = trow[i + 3], w = wr[i];
                s0 = fmaf(w, v0, s0);
                s1 = fmaf(w, v1, s1);
                s2 = fmaf(w, v2, s2);
                s3 = fmaf(w, v3, s3);
                v0 = v1;
                v1 = v2;
                v2 = v3;
            }
        }
    const int y = blockIdx.y * kTY + ty, z = blockIdx.z * kTZ + tz;
    if (y >= a.ny || z >= a.nz) return;
    const float sv[kXR] = {s0, s1, s2, s3};
#pragma unroll
    for (int c = 0; c < kXR; ++c) {
        const int x = blockIdx.x * kOX + kXR * g + c;
        if (x >= a.nx) continue;
        const long long o = ((long long)z * a.ny + y) * a.nx + x;
        float s = sv[c];
        if (a.div) s /= a.div[o];
        a.out[o] = s;
        if (a.proj) a.proj[o] = (tanhf(a.beta * a.eta) + tanhf(a.beta * (s - a.eta))) / a.pden;
    }
}

// Normalising sum of every voxel: the weights of the sphere's offsets (dx, dy, dz) whose target lies in
// the box, i.e. dx in [-min(x, n), min(nx-1-x, n)] and likewise in y, z, from the summed-volume table
// T[c][b][a] = sum of w over dz < c, dy < b, dx < a (offsets from -n) by inclusion-exclusion (FP64).
__global__ void wsum_kernel(const double* __restrict__ T, float* out, int nx, int ny, int nz, int n)
{
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= (long long)nx * ny * nz) return;
    const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long long)nx * ny));
    const int E = 2 * n + 2;                  // table extent per axis
    const int a0 = n - min(x, n), a1 = n + min(nx - 1 - x, n) + 1;
    const int b0 = n - min(y, n), b1 = n + min(ny - 1 - y, n) + 1;
    const int c0 = n - min(z, n), c1 = n + min(nz - 1 - z, n) + 1;
    auto t = [&](int c, int b, int a) { return __ldg(T + ((long long)c * E + b) * E + a); };
    const double s = t(c1, b1, a1) - t(c0, b1, a1) - t(c1, b0, a1) - t(c1, b1, a0) + t(c0, b0, a1) + t(c0, b1, a0) +
                     t(c1, b0, a0) - t(c0, b0, a0);
    out[v] = (float)s;
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
    const int n = a.n, W = 2 * n + 1;
    a.ntaps = 0;
    for (int dz = -n; dz <= n; ++dz)   // the same float test as the kernel's
        for (int dy = -n; dy <= n; ++dy)
            for (int dx = -n; dx <= n; ++dx) {
                bool inside;
                cone_weight(dx, dy, dz, a.R, inside);
                a.ntaps += inside ? 1 : 0;
            }
    const int Lx = kOX + 2 * n, Ly = kTY + 2 * n, Lz = kTZ + 2 * n;
    const size_t smem = sizeof(float) * ((size_t)Lz * Ly * row_pitch(Lx) + (size_t)a.ntaps) + sizeof(int) * 3 * (size_t)(W * W);
    cudaError_t e = cudaFuncSetAttribute(cone_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 g((nx + kOX - 1) / kOX, (ny + kTY - 1) / kTY, (nz + kTZ - 1) / kTZ);
    cone_kernel<<<g, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

// Normalising sums: the summed-volume table of the cone weights (the kernel's float weights, summed in
// FP64 on the host) and wsum_kernel.  T is a device buffer of (2n+2)^3 doubles.
cudaError_t norm_sums(float* out, double* T, int nx, int ny, int nz, double R, cudaStream_t s)
{
    const int n = (int)std::ceil(R) - 1, E = 2 * n + 2;
    std::vector<double> h((size_t)E * E * E, 0.0);
    for (int c = 1; c < E; ++c)
        for (int b = 1; b < E; ++b)
            for (int a = 1; a < E; ++a) {
                bool inside;
                const float w = cone_weight(a - 1 - n, b - 1 - n, c - 1 - n, (float)R, inside);
                const auto at = [&](int cc, int bb, int aa) { return h[((size_t)cc * E + bb) * E + aa]; };
                h[((size_t)c * E + b) * E + a] = (inside ? (double)w : 0.0) + at(c - 1, b, a) + at(c, b - 1, a) +
                                                  at(c, b, a - 1) - at(c - 1, b - 1, a) - at(c - 1, b, a - 1) -
                                                  at(c, b - 1, a - 1) + at(c - 1, b - 1, a - 1);
            }
    cudaError_t e = cudaMemcpyAsync(T, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    const long long nv = (long long)nx * ny * nz;
    wsum_kernel<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(T, out, nx, ny, nz, n);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the table's host copy lives on this stack
    return e;
}

size_t table_bytes(double R)
{
    const size_t E = 2 * ((size_t)std::ceil(R) - 1) + 2;
    return E * E * E * sizeof(double);
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
    cudaError_t e = cudaMallocAsync((void**)&Wsum, nv * sizeof(float) + table_bytes(R) + 256, s);
    if (e != cudaSuccess) return fail(FDTD_ERR_OOM, std::string("filter: ") + cudaGetErrorString(e));
    double* T = (double*)(((uintptr_t)(Wsum + nv) + 255) & ~(uintptr_t)255);
    e = norm_sums(Wsum, T, nx, ny, nz, R, s);                                                // normalising sums
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
    cudaError_t e = cudaMallocAsync((void**)&buf, 2 * nv * sizeof(float) + table_bytes(R) + 256, s);
    if (e != cudaSuccess) return fail(FDTD_ERR_OOM, std::string("filter grad: ") + cudaGetErrorString(e));
    float* Wsum = buf;
    float* g = buf + nv;
    double* T = (double*)(((uintptr_t)(buf + 2 * nv) + 255) & ~(uintptr_t)255);
    const float pden = (float)(std::tanh(beta * eta) + std::tanh(beta * (1.0 - eta)));
    e = norm_sums(Wsum, T, nx, ny, nz, R, s);
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
