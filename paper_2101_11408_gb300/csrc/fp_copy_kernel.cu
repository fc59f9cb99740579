// fp_copy_kernel.cu -- host <-> device data movement of the request server,
// done by kernels that read and write pinned host memory directly (the
// GPU reaches host memory over the CPU-GPU link; one kernel per batch
// replaces one copy call per request, whose fixed cost dominates small
// requests).
//
//   gather_kernel   copy pieces (src, dst, nbytes) -- the texts of a batch,
//                   host -> arena;
//   scatter_kernel  copy each request's first min(count, cap) values and
//                   statuses, arena -> host, reading count on the device, in
//                   pieces of at most SCATTER_PIECE fields.
// Piece tables live in pinned host memory and are read by the kernels.
#include <cuda_runtime.h>

#include <cstdint>

#include "fp_copy.h"

namespace fp {

namespace {

constexpr int COPY_NT = 256;

// Copy n bytes; src and dst have the same address modulo 16 (the server
// places each text so), so the body moves in 16-byte words.
__device__ __forceinline__ void copy_bytes(const uint8_t* src, uint8_t* dst, uint32_t n) {
  const uint32_t head = (uint32_t)((16 - ((uintptr_t)src & 15)) & 15);
  const uint32_t h = head < n ? head : n;
  if (threadIdx.x < h) dst[threadIdx.x] = src[threadIdx.x];
  const uint32_t body = (n - h) / 16;
  const uint4* s4 = reinterpret_cast<const uint4*>(src + h);
  uint4* d4 = reinterpret_cast<uint4*>(dst + h);
  for (uint32_t i = threadIdx.x; i < body; i += blockDim.x) d4[i] = s4[i];
  const uint32_t tail0 = h + 16 * body;
  for (uint32_t i = tail0 + threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

__global__ void __launch_bounds__(COPY_NT) gather_kernel(const CopyPiece* pieces, uint32_t npieces) {
  for (uint32_t k = blockIdx.x; k < npieces; k += gridDim.x) {
    const CopyPiece pc = pieces[k];
    if (((uintptr_t)pc.src ^ (uintptr_t)pc.dst) & 15) {  // not placed alike: bytes
      for (uint32_t i = threadIdx.x; i < pc.nbytes; i += blockDim.x) pc.dst[i] = pc.src[i];
    } else {
      copy_bytes(pc.src, pc.dst, pc.nbytes);
    }
  }
}

__global__ void __launch_bounds__(COPY_NT) scatter_kernel(const ScatterItem* items,
                                                          const ScatterPiece* pieces,
                                                          uint32_t npieces) {
  for (uint32_t k = blockIdx.x; k < npieces; k += gridDim.x) {
    const ScatterPiece pc = pieces[k];
    const ScatterItem it = items[pc.item];
    const unsigned long long count = *it.count;
    const unsigned long long n = count < it.cap ? count : it.cap;
    if (pc.first >= n) continue;
    const unsigned long long m0 = n - pc.first;
    const uint32_t m = m0 < SCATTER_PIECE ? (uint32_t)m0 : SCATTER_PIECE;
    const unsigned long long* sv = it.d_vals + pc.first;
    unsigned long long* dv = it.h_vals + pc.first;
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) dv[i] = sv[i];
    const uint8_t* ss = it.d_status + pc.first;
    uint8_t* ds = it.h_status + pc.first;
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) ds[i] = ss[i];
  }
}

}  // namespace

cudaError_t launch_gather(const CopyPiece* pieces, uint32_t npieces, int grid,
                          cudaStream_t stream) {
  if (npieces == 0) return cudaSuccess;
  gather_kernel<<<grid, COPY_NT, 0, stream>>>(pieces, npieces);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const ScatterItem* items, const ScatterPiece* pieces, uint32_t npieces,
                           int grid, cudaStream_t stream) {
  if (npieces == 0) return cudaSuccess;
  scatter_kernel<<<grid, COPY_NT, 0, stream>>>(items, pieces, npieces);
  return cudaGetLastError();
}

}  // namespace fp
