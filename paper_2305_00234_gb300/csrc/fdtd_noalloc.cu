// fdtd_gradient_static: the per-voxel gradient reduction with its scratch memory in a static
// device array, for callers that must not allocate device memory (see include/fdtd_ccpr.h).
//
// The kernel is the library's grad_kernel; only where its scratch lives differs.  Scratch layout
// inside g_scratch (kScratchBytes, 256-byte aligned):
//   [0, 1024)        dY/drho constants, 3 components x up to 8 frequencies x (A, B) as double2
//   [1024, 1280)     block-completion counter (unsigned)
//   [1280, end)      per-block partial sums of grad^2 and their total (doubles)
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "fdtd_ccpr.h"
#include "fdtd_kernels.cuh"

namespace fdtd {
void set_thread_error(const std::string& msg);
}

namespace {

constexpr size_t kScratchBytes = 1u << 20;
constexpr size_t kConstOffset = 0;
constexpr size_t kCounterOffset = 1024;
constexpr size_t kPartialOffset = 1280;
constexpr size_t kMaxPartials = (kScratchBytes - kPartialOffset) / sizeof(double);   // blocks + 1 total
constexpr long long kMaxDesignVoxels = (long long)(kMaxPartials - 1) * fdtd::kReduceThreads;
constexpr int kMaxDevices = 64;

// One copy per device that loads the library, held until process exit.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

fdtd_status fail(fdtd_status code, const std::string& msg)
{
    fdtd::set_thread_error("fdtd_gradient_static: " + msg);
    return code;
}

// Device address of g_scratch on the current device, looked up once per device.  The host-side
// name g_scratch is only a stand-in for the symbol, never a pointer a kernel may use.
fdtd_status scratch_address(int device, unsigned char** out)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return fail(FDTD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[device] = p;
    }
    *out = (unsigned char*)g_scratch_addr[device];
    return FDTD_OK;
}

bool box_ok(const int* b) { return b[0] < b[1] && b[2] < b[3] && b[4] < b[5] && b[0] >= 0 && b[2] >= 0 && b[4] >= 0; }

template <typename T>
cudaError_t launch(const double* df, const double* da, const void* rho, const int* db, const int* gb, int nf,
                   unsigned char* scratch, double* grad, cudaStream_t s, unsigned nblocks)
{
    fdtd::GParams<T> g{};
    for (int q = 0; q < 6; ++q) {
        g.db[q] = db[q];
        g.gb[q] = gb ? gb[q] : 0;
    }
    g.dnx = db[1] - db[0];
    g.dny = db[3] - db[2];
    g.nd = (long long)g.dnx * g.dny * (db[5] - db[4]);
    g.nf = nf;
    g.dft_f = (const double2*)df;
    g.dft_a = (const double2*)da;
    g.AB = (const double2*)(scratch + kConstOffset);
    g.rho = (const T*)rho;
    g.grad64 = grad;
    g.grad32 = nullptr;
    g.partial = (double*)(scratch + kPartialOffset);
    g.counter = (unsigned*)(scratch + kCounterOffset);
    fdtd::grad_kernel<T><<<nblocks, fdtd::kReduceThreads, 0, s>>>(g);
    return cudaGetLastError();
}

}  // namespace

extern "C" fdtd_status fdtd_gradient_static(const double* dft_fwd, const double* dft_adj, const void* rho,
                                            int rho_dtype, const int design_box[6], const int gap_box[6],
                                            int n_freq, const double* dy_drho, double* grad,
                                            double* grad_norm2, void* cuda_stream)
{
    if (!dft_fwd || !dft_adj || !rho || !design_box || !dy_drho || !grad)
        return fail(FDTD_ERR_ARG, "null pointer argument");
    if (rho_dtype != 0 && rho_dtype != 1) return fail(FDTD_ERR_ARG, "rho_dtype must be 0 (float32) or 1 (float64)");
    if (n_freq < 1 || n_freq > fdtd::kMaxFreq) return fail(FDTD_ERR_ARG, "n_freq must be in [1, 8]");
    if (!box_ok(design_box)) return fail(FDTD_ERR_ARG, "empty or negative design box");
    const bool has_gap = gap_box && gap_box[0] < gap_box[1] && gap_box[2] < gap_box[3] && gap_box[4] < gap_box[5];
    const long long nd = (long long)(design_box[1] - design_box[0]) * (design_box[3] - design_box[2]) *
                         (design_box[5] - design_box[4]);
    if (nd > kMaxDesignVoxels)
        return fail(FDTD_ERR_ARG, "design box has " + std::to_string(nd) + " voxels; the static scratch holds partial "
                                  "sums for at most " + std::to_string(kMaxDesignVoxels));
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return fail(FDTD_ERR_CUDA, cudaGetErrorString(e));
    if (device < 0 || device >= kMaxDevices) return fail(FDTD_ERR_ARG, "device ordinal above 63");
    unsigned char* scratch = nullptr;
    if (fdtd_status st = scratch_address(device, &scratch)) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // constants (A, B) as double2 pairs, and a zeroed counter: the array keeps the last call's bytes
    e = cudaMemcpyAsync(scratch + kConstOffset, dy_drho, 3 * (size_t)n_freq * 4 * sizeof(double),
                        cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch + kCounterOffset, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return fail(FDTD_ERR_CUDA, cudaGetErrorString(e));
    const int none[6] = {0, 0, 0, 0, 0, 0};
    const unsigned nblocks = (unsigned)((nd + fdtd::kReduceThreads - 1) / fdtd::kReduceThreads);
    e = rho_dtype == 0 ? launch<float>(dft_fwd, dft_adj, rho, design_box, has_gap ? gap_box : none, n_freq, scratch,
                                       grad, s, nblocks)
                       : launch<double>(dft_fwd, dft_adj, rho, design_box, has_gap ? gap_box : none, n_freq, scratch,
                                        grad, s, nblocks);
    if (e != cudaSuccess) return fail(FDTD_ERR_CUDA, cudaGetErrorString(e));
    if (grad_norm2) {
        e = cudaMemcpyAsync(grad_norm2, scratch + kPartialOffset + nblocks * sizeof(double), sizeof(double),
                            cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(FDTD_ERR_CUDA, cudaGetErrorString(e));
    }
    return FDTD_OK;
}
