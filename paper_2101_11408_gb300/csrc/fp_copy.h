// fp_copy.h -- copy kernels (fp_copy_kernel.cu): the request server's
// gather and scatter, and the packing of a batch's results.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace fp {

// One piece of a host -> device gather: nbytes from src (a host address the
// device can reach) to dst (device memory).
struct CopyPiece {
  const uint8_t* src;
  uint8_t* dst;
  uint32_t nbytes;
  uint32_t pad;
};
constexpr uint32_t GATHER_PIECE = 256u << 10;  // bytes per piece at most

// One request of a device -> host scatter: its first min(*count, cap)
// values and statuses.
struct ScatterItem {
  const unsigned long long* d_vals;
  const uint8_t* d_status;
  unsigned long long* h_vals;
  uint8_t* h_status;
  const unsigned long long* count;  // device
  unsigned long long cap;
};
// A piece: fields [first, first + SCATTER_PIECE) of one item.
struct ScatterPiece {
  uint32_t item;
  uint32_t pad;
  unsigned long long first;
};
constexpr uint32_t SCATTER_PIECE = 32768;  // fields per piece at most

// Packing of a batch's results: buffer b owns output entries [bases[b],
// bases[b + 1]) (nbuf + 1 offsets) and keeps kept_b = min(counts[b],
// bases[b + 1] - bases[b]) results there; they go to dst at the sum of the
// earlier buffers' kept_b.  A piece is (b << 40) | f0: fields [f0, f0 +
// PACK_PIECE) of buffer b's capacity.
constexpr uint32_t PACK_PIECE = 8192;  // fields per piece at most
// starts[b] = sum of kept_b' for b' < b (b <= nbuf; starts[nbuf] is the
// total, also written to *total when total is not null); one block.
cudaError_t launch_pack_scan(const unsigned long long* counts, const unsigned long long* bases,
                             uint32_t nbuf, unsigned long long* starts, unsigned long long* total,
                             cudaStream_t stream);
cudaError_t launch_pack_copy(const unsigned long long* pieces, unsigned long long npieces,
                             const unsigned long long* counts,
                             const unsigned long long* bases, const unsigned long long* starts,
                             const unsigned long long* src_vals, const uint8_t* src_status,
                             unsigned long long* dst_vals, uint8_t* dst_status, int grid,
                             cudaStream_t stream);

cudaError_t launch_gather(const CopyPiece* pieces, uint32_t npieces, int grid, cudaStream_t stream);
cudaError_t launch_scatter(const ScatterItem* items, const ScatterPiece* pieces, uint32_t npieces,
                           int grid, cudaStream_t stream);

}  // namespace fp
