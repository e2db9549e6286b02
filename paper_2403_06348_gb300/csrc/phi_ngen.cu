// Phi kernels (CP-APR, Alg. 5) for any other number of modes (decided at run time).
#include "mttkrp_kernel.cuh"

namespace alto {
template cudaError_t launch_phi_nt<0>(const MttkrpArgs &, bool, bool, size_t, int, cudaStream_t);
}  // namespace alto
