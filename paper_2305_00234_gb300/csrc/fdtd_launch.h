// Host-side declarations of the kernel launch wrappers (defined in fdtd_kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fdtd_params.h"

namespace fdtd {

int pole_bucket(int max_poles);
template <typename T>
cudaError_t prepare_step();
// pdl: launch as a programmatic dependent launch in the step chain (see pdl_wait in fdtd_kernels.cuh)
template <typename T>
unsigned step_blocks(const KParams<T>& p);
// kernel nodes of a step graph, without dependencies
template <typename T>
cudaError_t graph_step(cudaGraph_t g, cudaGraphNode_t* node, const KParams<T>& p, const StepMaps& m);
template <typename T>
cudaError_t graph_shell(cudaGraph_t g, cudaGraphNode_t* node, const KParams<T>& p, const ShellBoxes& s, bool e_part);
template <typename T>
cudaError_t graph_e_design(cudaGraph_t g, cudaGraphNode_t* node, const KParams<T>& p, const PoleTable<T>& tab, int bucket);
template <typename T>
cudaError_t graph_dft(cudaGraph_t g, cudaGraphNode_t* node, const DParams<T>& d, int cnt);
template <typename T>
cudaError_t launch_step(const KParams<T>& p, const StepMaps& m, cudaStream_t s, bool pdl = false);
template <typename T>
cudaError_t launch_e_design(const KParams<T>& p, const PoleTable<T>& tab, int bucket, cudaStream_t s, bool pdl = false);
template <typename T>
cudaError_t launch_dft(const DParams<T>& d, int cnt, cudaStream_t s, bool pdl = false);
unsigned shell_blocks(ShellBoxes& s);   // fills s.first, returns the launch's blocks
template <typename T>
cudaError_t launch_shell(const KParams<T>& p, const ShellBoxes& s, bool e_part, cudaStream_t st, bool pdl = false);
unsigned design_blocks(int dnx, int dny, int dnz, int& edz, bool flat);   // also picks the column depth
template <typename T>
cudaError_t launch_grad(const GParams<T>& g, unsigned nblocks, cudaStream_t s);
cudaError_t launch_gap_gather(const double2* dft, long long nd, int nf, const int* db, int dnx, int dny, const int* gb,
                              double2* out, cudaStream_t s);
template <typename T>
cudaError_t launch_rho_import(const void* src, int dtype, long long n, T* dst, int* flag, cudaStream_t s);
template <typename T>
cudaError_t launch_rho_scatter(const void* src, int dtype, long long n, const long long off[4], const int md[3][3],
                               int dnx, int dny, long long nd, T* dst, int* flag, cudaStream_t s);
template <typename T>
cudaError_t launch_to_double(const T* src, long long n, double* dst, cudaStream_t s);
template <typename T>
cudaError_t launch_gather_design_e(const KParams<T>& p, T* out, cudaStream_t s);
template <typename T>
cudaError_t launch_paper_drive(const T* gh, T* drive, int M, int ns, double eps0, cudaStream_t s);
template <typename T>
cudaError_t launch_paper_grad(const PParams<T>& g, cudaStream_t s);
template <typename T>
cudaError_t launch_index_map(const KParams<T>& p, int which, int32_t* out, cudaStream_t s);
// persistent batch kernel (fdtd_batch.cu): its function for a pole bucket, and resident blocks per SM
template <typename T>
const void* batch_kernel_fn(int bucket);
template <typename T>
cudaError_t batch_blocks_per_sm(int bucket, int* out);

}  // namespace fdtd
