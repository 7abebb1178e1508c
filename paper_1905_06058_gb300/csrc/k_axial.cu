// Instances of the axial Stolt-mapped NUFFT kernels (k_axial.cuh) for the
// FP32 plans; the two precisions compile as separate units, in parallel.
#include "k_axial.cuh"

namespace isam {

template cudaError_t launch_stolt_table<float>(const AxArgs<float>&, StoltEntry<float>*, cudaStream_t);
template size_t ax_smem_bytes<float>(int, int, bool);
template cudaError_t launch_ax_fwd<float>(const AxArgs<float>&, int, cudaStream_t);
template cudaError_t launch_ax_adj<float>(const AxArgs<float>&, int, cudaStream_t);
template cudaError_t launch_ax_fused<float>(const AxArgs<float>&, int, cudaStream_t);

}  // namespace isam
