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
//   pack_scan_kernel / pack_copy_kernel  a batch's results packed in buffer
//                   order (device to device): an exclusive scan of the
//                   per-buffer counts, then fixed-size pieces of each
//                   buffer's output range copied to their packed place.
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

constexpr int SCAN_NT = 1024;

// The results buffer b holds: its count, at most its output capacity (a
// buffer with more fields than room keeps only the first ones).
__device__ __forceinline__ unsigned long long kept(const unsigned long long* counts,
                                                   const unsigned long long* bases, uint32_t b) {
  const unsigned long long cap = bases[b + 1] - bases[b];
  return counts[b] < cap ? counts[b] : cap;
}

__global__ void __launch_bounds__(SCAN_NT) pack_scan_kernel(const unsigned long long* counts,
                                                            const unsigned long long* bases,
                                                            uint32_t nbuf,
                                                            unsigned long long* starts,
                                                            unsigned long long* total) {
  __shared__ unsigned long long wsum[SCAN_NT / 32];
  const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // thread t sums buffers [t * per, (t + 1) * per)
  const uint32_t per = (nbuf + SCAN_NT - 1) / SCAN_NT;
  const uint32_t b0 = t * per, b1 = min(b0 + per, nbuf);
  unsigned long long mine = 0;
  for (uint32_t b = b0; b < b1; b++) mine += kept(counts, bases, b);
  unsigned long long incl = mine;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, incl, off);
    if (lane >= off) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  unsigned long long before = 0, all = 0;
  for (int w = 0; w < SCAN_NT / 32; w++) {
    before += w < (int)warp ? wsum[w] : 0ull;
    all += wsum[w];
  }
  unsigned long long run = before + incl - mine;  // exclusive prefix of this thread's first buffer
  for (uint32_t b = b0; b < b1; b++) {
    starts[b] = run;
    run += kept(counts, bases, b);
  }
  if (t == 0) {
    starts[nbuf] = all;
    if (total) *total = all;
  }
}

__global__ void __launch_bounds__(COPY_NT) pack_copy_kernel(
    const unsigned long long* pieces, unsigned long long npieces,
    const unsigned long long* counts, const unsigned long long* bases,
    const unsigned long long* starts, const unsigned long long* src_vals,
    const uint8_t* src_status, unsigned long long* dst_vals, uint8_t* dst_status) {
  for (unsigned long long k = blockIdx.x; k < npieces; k += gridDim.x) {
    const unsigned long long pc = pieces[k];
    const uint32_t b = (uint32_t)(pc >> 40);
    const unsigned long long f0 = pc & ((1ull << 40) - 1);
    const unsigned long long count = kept(counts, bases, b);
    if (f0 >= count) continue;
    const unsigned long long m0 = count - f0;
    const uint32_t m = m0 < PACK_PIECE ? (uint32_t)m0 : PACK_PIECE;
    const unsigned long long* sv = src_vals + bases[b] + f0;
    const uint8_t* ss = src_status + bases[b] + f0;
    unsigned long long* dv = dst_vals + starts[b] + f0;
    uint8_t* ds = dst_status + starts[b] + f0;
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) dv[i] = sv[i];
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) ds[i] = ss[i];
  }
}

}  // namespace

cudaError_t launch_pack_scan(const unsigned long long* counts, const unsigned long long* bases,
                             uint32_t nbuf, unsigned long long* starts, unsigned long long* total,
                             cudaStream_t stream) {
  pack_scan_kernel<<<1, SCAN_NT, 0, stream>>>(counts, bases, nbuf, starts, total);
  return cudaGetLastError();
}

cudaError_t launch_pack_copy(const unsigned long long* pieces, unsigned long long npieces,
                             const unsigned long long* counts,
                             const unsigned long long* bases, const unsigned long long* starts,
                             const unsigned long long* src_vals, const uint8_t* src_status,
                             unsigned long long* dst_vals, uint8_t* dst_status, int grid,
                             cudaStream_t stream) {
  if (npieces == 0) return cudaSuccess;
  pack_copy_kernel<<<grid, COPY_NT, 0, stream>>>(pieces, npieces, counts, bases, starts, src_vals,
                                                 src_status, dst_vals, dst_status);
  return cudaGetLastError();
}

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
