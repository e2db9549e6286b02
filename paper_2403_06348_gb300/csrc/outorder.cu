// The stored output-oriented order pos_out of Alg. 4 and the dispatch of its
// MTTKRP kernel by number of modes (kernels in outorder.cuh, out_n*.cu).
//
// pos_out of a mode is built as one stable LSD radix sort of the whole line:
// the key of ordered position x is (segment of x, coordinate of the mode) and
// the sorted values are the positions themselves. Segments are contiguous and
// the sort is stable, so this is the per-segment stable sort by coordinate.
#include "encode.cuh"
#include "handle.cuh"
#include "outorder.cuh"

namespace alto {

// key[x] = l(x) << bits | i_mode(x), pos[x] = x, where l(x) is the segment
// [floor(l M / L), floor((l + 1) M / L)) holding x: l(x) = floor(((x + 1) L - 1) / M).
template <int KW>
__global__ void __launch_bounds__(256) pos_key_kernel(const __grid_constant__ DecodePlan dp,
                                                      const uint64_t *__restrict__ keys, uint64_t nnz,
                                                      uint64_t L, int mode, int bits,
                                                      uint64_t *__restrict__ ck,
                                                      uint32_t *__restrict__ pos) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nnz;
       x += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t c[kMaxModes];
    decode_all<KW>(dp, keys[x * KW], KW == 2 ? keys[x * KW + 1] : 0ull, c);
    uint32_t i = 0;
#pragma unroll
    for (int n = 0; n < kMaxModes; ++n)
      if (n == mode) i = c[n];
    const uint64_t l = ((x + 1) * L - 1) / nnz;
    ck[x] = (l << bits) | i;
    pos[x] = (uint32_t)x;
  }
}

static int bit_width_u64(uint64_t v) {
  int b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

alto_status build_pos_out(alto_tensor *h, int mode, uint64_t L, uint32_t **out, cudaStream_t s) {
  *out = nullptr;
  const uint64_t M = h->M;
  if (M > kPosOutMaxNnz)
    return fail(ALTO_ERR_UNSUPPORTED, "pos_out holds 32-bit positions: nnz %llu too large",
                (unsigned long long)M);
  if (L < 1 || L > M) L = M ? std::min<uint64_t>(std::max<uint64_t>(L, 1), M) : 1;
  const int bits = h->bits[mode];
  const int nbits = bit_width_u64(L - 1) + bits;  // <= 32 + 32
  uint64_t *kbuf[2] = {nullptr, nullptr};
  float *vbuf[2] = {nullptr, nullptr};
  uint32_t *pos = nullptr, *table = nullptr, *table_scan = nullptr, *block_sums = nullptr;
  const size_t entries = sort_table_entries(M);
  const size_t nblocks = std::max<size_t>(sort_scan_blocks(M), 1);
  auto release = [&](int keep) {
    for (int b = 0; b < 2; ++b) {
      dfree(h, kbuf[b], M * 8, s);
      if (b != keep) dfree(h, vbuf[b], M * 4, s);
    }
    dfree(h, pos, M * 4, s);
    dfree(h, table, entries * 4, s);
    dfree(h, table_scan, entries * 4, s);
    dfree(h, block_sums, nblocks * 4, s);
  };
  uint32_t *res = static_cast<uint32_t *>(dalloc(h, std::max<uint64_t>(M, 1) * 4, s));
  if (!res) return fail(ALTO_ERR_OOM, "pos_out of %llu entries", (unsigned long long)M);
  if (M == 0) {
    *out = res;
    return ALTO_OK;
  }
  for (int b = 0; b < 2; ++b) {
    kbuf[b] = static_cast<uint64_t *>(dalloc(h, M * 8, s));
    vbuf[b] = b == 0 ? reinterpret_cast<float *>(res) : static_cast<float *>(dalloc(h, M * 4, s));
  }
  pos = static_cast<uint32_t *>(dalloc(h, M * 4, s));
  table = static_cast<uint32_t *>(dalloc(h, entries * 4, s));
  table_scan = static_cast<uint32_t *>(dalloc(h, entries * 4, s));
  block_sums = static_cast<uint32_t *>(dalloc(h, nblocks * 4, s));
  if (!kbuf[0] || !kbuf[1] || !vbuf[1] || !pos || !table || !table_scan || !block_sums) {
    release(-1);
    return fail(ALTO_ERR_OOM, "pos_out sort scratch for %llu entries", (unsigned long long)M);
  }
  const int grid = (int)std::min<uint64_t>((M + 255) / 256, (uint64_t)h->num_sms * 8);
  if (h->kw == 1)
    pos_key_kernel<1><<<grid, 256, 0, s>>>(h->dp, h->keys, M, L, mode, bits, kbuf[0], pos);
  else
    pos_key_kernel<2><<<grid, 256, 0, s>>>(h->dp, h->keys, M, L, mode, bits, kbuf[0], pos);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  int fbuf = 0;
  // the positions travel through the sort as 32-bit payload words, bit for bit
  if (e == cudaSuccess)
    e = launch_radix_sort(1, nbits, M, kbuf, vbuf, reinterpret_cast<const float *>(pos), table,
                          table_scan, block_sums, &fbuf, s);
  if (e != cudaSuccess) {
    release(-1);
    return fail(ALTO_ERR_CUDA, "pos_out: %s", cudaGetErrorString(e));
  }
  if (fbuf == 0) {
    release(0);
  } else {
    // result in vbuf[1]: keep it, free the buffer that was allocated as res
    dfree(h, res, M * 4, s);
    vbuf[0] = nullptr;
    res = reinterpret_cast<uint32_t *>(vbuf[1]);
    release(1);
  }
  *out = res;
  return ALTO_OK;
}

cudaError_t launch_mttkrp_out(const MttkrpArgs &a, int cpl, bool bf16, int num_sms, cudaStream_t s) {
  if (a.nnz == 0) return cudaSuccess;
  switch (a.dp.nmodes) {
    case 3: return launch_mttkrp_out_nt<3>(a, cpl, bf16, num_sms, s);
    case 4: return launch_mttkrp_out_nt<4>(a, cpl, bf16, num_sms, s);
    case 5: return launch_mttkrp_out_nt<5>(a, cpl, bf16, num_sms, s);
    default: return launch_mttkrp_out_nt<0>(a, cpl, bf16, num_sms, s);
  }
}

}  // namespace alto
