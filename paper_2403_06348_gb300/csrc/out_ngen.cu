// Output-oriented MTTKRP and Phi kernels for any number of modes (decided at run time).
#include "outorder.cuh"

namespace alto {
template cudaError_t launch_mttkrp_out_nt<0>(const MttkrpArgs &, int, bool, size_t, int, cudaStream_t);
template cudaError_t launch_phi_out_nt<0>(const MttkrpArgs &, bool, size_t, int, cudaStream_t);
}  // namespace alto
