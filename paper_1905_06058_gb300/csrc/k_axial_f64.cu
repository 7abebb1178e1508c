// Instances of the axial Stolt-mapped NUFFT kernels (k_axial.cuh) for the
// FP64 plans; the two precisions compile as separate units, in parallel.
#include "k_axial.cuh"

namespace isam {

template cudaError_t launch_stolt_table<double>(const AxArgs<double>&, StoltEntry<double>*, cudaStream_t);
template size_t ax_smem_bytes<double>(int, int, bool);
template cudaError_t launch_ax_fwd<double>(const AxArgs<double>&, int, cudaStream_t);
template cudaError_t launch_ax_adj<double>(const AxArgs<double>&, int, cudaStream_t);
template cudaError_t launch_ax_fused<double>(const AxArgs<double>&, int, cudaStream_t);

}  // namespace isam
