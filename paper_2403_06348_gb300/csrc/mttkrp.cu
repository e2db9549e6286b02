// MTTKRP host dispatch and the pull-based reduction of Alg. 4. The segment
// kernel itself is in mttkrp_kernel.cuh, instantiated per mode count by
// mttkrp_n*.cu.
#include "mttkrp.cuh"

namespace alto {

// out(b,:) = sum over segments l with b in [T^s_l, T^e_l] of Temp_l(b - T^s_l, :)
// (Alg. 4, pull-based reduction); prow lists, per row, the partial rows to add.
__global__ void __launch_bounds__(256) pull_reduce_kernel(const float *__restrict__ partials,
                                                          const uint64_t *__restrict__ row_ptr,
                                                          const uint64_t *__restrict__ prow,
                                                          uint64_t I, int R, float *__restrict__ out,
                                                          const int *__restrict__ skip) {
  if (skip && *skip) return;
  const int per_row = R / 4;
  const uint64_t total = I * (uint64_t)per_row;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = t / per_row;
    const int c4 = (int)(t - b * per_row) * 4;
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (uint64_t e = row_ptr[b]; e < row_ptr[b + 1]; ++e) {
      const float4 p = *reinterpret_cast<const float4 *>(partials + prow[e] * (uint64_t)R + c4);
      s0 += p.x;
      s1 += p.y;
      s2 += p.z;
      s3 += p.w;
    }
    *reinterpret_cast<float4 *>(out + b * (uint64_t)R + c4) =
        make_float4((float)s0, (float)s1, (float)s2, (float)s3);
  }
}

size_t mttkrp_smem_bytes(bool pull, int R, int nslots, int hbits, uint32_t max_interval) {
  if (pull) return (size_t)max_interval * (size_t)R * sizeof(float);
  return (size_t)nslots * R * sizeof(float) + ((size_t)1 << hbits) * sizeof(uint64_t);
}

size_t mttkrp_smem_limit() {
  static int v = 0;
  if (!v) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  return (size_t)v;
}

size_t mttkrp_stage_budget() {
  static int per_sm = 0;
  if (!per_sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  }
  size_t b = (size_t)per_sm / kMttkrpBlocksPerSm - 2048;
  return b < mttkrp_smem_limit() ? b : mttkrp_smem_limit();
}

cudaError_t launch_mttkrp(const MttkrpArgs &a, int cpl, bool bf16, bool pull, size_t smem,
                          int num_sms, cudaStream_t s) {
  if (a.nnz == 0) return cudaSuccess;
  switch (a.dp.nmodes) {
    case 3: return launch_mttkrp_nt<3>(a, cpl, bf16, pull, smem, num_sms, s);
    case 4: return launch_mttkrp_nt<4>(a, cpl, bf16, pull, smem, num_sms, s);
    case 5: return launch_mttkrp_nt<5>(a, cpl, bf16, pull, smem, num_sms, s);
    default: return launch_mttkrp_nt<0>(a, cpl, bf16, pull, smem, num_sms, s);
  }
}

cudaError_t launch_pull_reduce(const float *partials, const uint64_t *row_ptr, const uint64_t *prow,
                               uint64_t I, int R, float *out, int num_sms, cudaStream_t s,
                               const int *skip) {
  const uint64_t total = I * (uint64_t)(R / 4);
  uint64_t grid = (total + 255) / 256;
  if (grid > (uint64_t)num_sms * 16) grid = (uint64_t)num_sms * 16;
  if (grid < 1) grid = 1;
  pull_reduce_kernel<<<(unsigned)grid, 256, 0, s>>>(partials, row_ptr, prow, I, R, out, skip);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_phi(const MttkrpArgs &a, bool pull, bool pre, size_t smem, int num_sms,
                       cudaStream_t s) {
  if (a.nnz == 0) return cudaSuccess;
  switch (a.dp.nmodes) {
    case 3: return launch_phi_nt<3>(a, pull, pre, smem, num_sms, s);
    case 4: return launch_phi_nt<4>(a, pull, pre, smem, num_sms, s);
    case 5: return launch_phi_nt<5>(a, pull, pre, smem, num_sms, s);
    default: return launch_phi_nt<0>(a, pull, pre, smem, num_sms, s);
  }
}

}  // namespace alto
