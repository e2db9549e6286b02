// In-tile output-oriented MTTKRP kernels for any number of modes (decided at
// run time), plus the dispatch by number of modes and the warm-row reduction.
#include "tile.cuh"

namespace alto {
template cudaError_t launch_mttkrp_tile_nt<0>(const MttkrpArgs &, int, bool, bool, int, cudaStream_t);

cudaError_t launch_mttkrp_tile(const MttkrpArgs &a, int cpl, bool bf16, bool group, int num_sms,
                               cudaStream_t s) {
  if (a.nnz == 0) return cudaSuccess;
  switch (a.dp.nmodes) {
    case 3: return launch_mttkrp_tile_nt<3>(a, cpl, bf16, group, num_sms, s);
    case 4: return launch_mttkrp_tile_nt<4>(a, cpl, bf16, group, num_sms, s);
    case 5: return launch_mttkrp_tile_nt<5>(a, cpl, bf16, group, num_sms, s);
    default: return launch_mttkrp_tile_nt<0>(a, cpl, bf16, group, num_sms, s);
  }
}

size_t tile_smem_bytes(int nmodes, int kw, int R, int cpl, int nslots, int hbits, int nbins, bool lut) {
  const int nmax = (nmodes == 3 || nmodes == 4 || nmodes == 5) ? nmodes : kMaxModes;
  const int rw = nmax + 1 <= 4 ? 4 : (nmax + 1 <= 8 ? 8 : 12);
  return tile_layout(kw, rw * 4, kTileThreads / (R / cpl), R, nslots, hbits, nbins, lut).total;
}

// One thread per 2 columns of a warm slot: the fp64 replicas summed in slot
// order, the row written in fp32 (every update of a warm row went to the
// replicas), the replicas cleared.
__global__ void __launch_bounds__(256) warm_reduce_kernel(double *__restrict__ warm,
                                                          const uint32_t *__restrict__ slot_rows,
                                                          int nslots, int nbins, int R,
                                                          float *__restrict__ out) {
  const int per_row = R / 2;
  const int total = (nbins - nslots) * per_row;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int slot = nslots + i / per_row, c2 = (i % per_row) * 2;
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll 4
    for (int g = 0; g < kWarmReps; ++g) {
      double2 *p = reinterpret_cast<double2 *>(warm + ((size_t)g * nbins + slot) * R + c2);
      const double2 v = *p;
      acc.x += v.x;
      acc.y += v.y;
      *p = make_double2(0.0, 0.0);
    }
    *reinterpret_cast<float2 *>(out + (uint64_t)slot_rows[slot] * R + c2) =
        make_float2((float)acc.x, (float)acc.y);
  }
}

cudaError_t launch_warm_reduce(double *warm, const uint32_t *slot_rows, int nslots, int nbins, int R,
                               float *out, int num_sms, cudaStream_t s) {
  const int total = (nbins - nslots) * (R / 2);
  if (total <= 0) return cudaSuccess;
  int grid = (total + 255) / 256;
  if (grid > num_sms * 4) grid = num_sms * 4;
  warm_reduce_kernel<<<grid, 256, 0, s>>>(warm, slot_rows, nslots, nbins, R, out);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace alto
