// MTTKRP segment kernels specialised for 5 modes.
#include "mttkrp_kernel.cuh"

namespace alto {
template cudaError_t launch_mttkrp_nt<5>(const MttkrpArgs &, int, bool, bool, size_t, int, cudaStream_t);
}  // namespace alto
