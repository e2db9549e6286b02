// MTTKRP segment kernels specialised for any number of modes (decided at run time).
#include "mttkrp_kernel.cuh"

namespace alto {
template cudaError_t launch_mttkrp_nt<0>(const MttkrpArgs &, int, bool, bool, size_t, int, cudaStream_t);
}  // namespace alto
