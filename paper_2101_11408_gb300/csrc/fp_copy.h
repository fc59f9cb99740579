// fp_copy.h -- the request server's copy kernels (fp_copy_kernel.cu).
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

cudaError_t launch_gather(const CopyPiece* pieces, uint32_t npieces, int grid, cudaStream_t stream);
cudaError_t launch_scatter(const ScatterItem* items, const ScatterPiece* pieces, uint32_t npieces,
                           int grid, cudaStream_t stream);

}  // namespace fp
