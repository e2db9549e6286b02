// MTTKRP segment kernels specialised for 3 modes.
#include "mttkrp_kernel.cuh"

namespace alto {
template cudaError_t launch_mttkrp_nt<3>(const MttkrpArgs &, int, bool, bool, size_t, int, cudaStream_t);
}  // namespace alto
