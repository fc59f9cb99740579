// fp_launch.h -- host-side entry points of the kernel translation units.
#pragma once
#include <cuda_runtime.h>

#include "fp_types.cuh"

namespace fp {

// f32: binary32 results (4-byte values; pending locations in p.loc),
// else binary64 (8-byte values; p.loc == p.out_bits).
cudaError_t launch_parse(const LaunchParams& p, int chunk_bytes, int grid, cudaStream_t stream,
                         bool f32 = false);
// The JSON / hexadecimal / column-major modes (mode: MODE_* bits of
// fp_parse_kernel.cuh, nonzero), for 8 KiB and 16 KiB chunks; the blocks
// per SM that every one of those instances reaches.
cudaError_t launch_parse_ext(const LaunchParams& p, int chunk_bytes, int grid,
                             cudaStream_t stream, bool f32, int mode);
cudaError_t parse_occupancy_ext(int chunk_bytes, int* blocks_per_sm);
cudaError_t parse_occupancy(int chunk_bytes, int* blocks_per_sm, bool f32 = false);

// The fallback kernel in two builds: for a launch expected to find nothing
// queued (the stream's last finished call had no fallback work: it reads the
// queue counters and returns), registers for FB_IDLE_BLOCKS per SM; for a
// stream with fallback work (busy), fewer registers and FB_BUSY_BLOCKS per SM.
constexpr int FB_IDLE_BLOCKS = 5;
constexpr int FB_BUSY_BLOCKS = 8;
cudaError_t launch_fallback(const LaunchParams& p, int grid, cudaStream_t stream, bool f32 = false,
                            bool busy = false);
cudaError_t fallback_occupancy(int* blocks_per_sm, bool f32 = false, bool busy = false);
// a one-block launch that separates the parse and fallback kernels (see
// fp_fallback_kernel.cu)
cudaError_t launch_fallback_separator(cudaStream_t stream);

}  // namespace fp
