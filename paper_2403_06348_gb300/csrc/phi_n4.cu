// Phi kernels (CP-APR, Alg. 5) for tensors with 4 modes.
#include "mttkrp_kernel.cuh"

namespace alto {
template cudaError_t launch_phi_nt<4>(const MttkrpArgs &, bool, bool, size_t, int, cudaStream_t);
}  // namespace alto
