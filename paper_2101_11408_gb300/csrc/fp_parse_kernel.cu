// fp_parse_kernel.cu -- the parse kernel's default-mode instances (binary64
// and binary32, decimal and hexadecimal grammars) and their launch helpers;
// the kernel itself is in fp_parse_kernel.cuh.
#include "fp_launch.h"
#include "fp_parse_kernel.cuh"

namespace fp {

template <int C, class F>
static cudaError_t launch_parse_c(const LaunchParams& p, int grid, cudaStream_t stream) {
  static bool attr_set = false;  // the attribute is per function; set it once
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(parse_kernel<C, F, 0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Layout<C>::TOTAL);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = Layout<C>::TOTAL;
  cfg.stream = stream;
  // a programmatic dependent launch (the kernel waits on the device for the
  // kernel before it; see parse_kernel)
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, parse_kernel<C, F, 0>, p);
}

template <class F>
static cudaError_t launch_parse_f(const LaunchParams& p, int chunk_bytes, int grid,
                                  cudaStream_t stream) {
  switch (chunk_bytes) {
    case 4096: return launch_parse_c<4096, F>(p, grid, stream);
    case 8192: return launch_parse_c<8192, F>(p, grid, stream);
    case 12288: return launch_parse_c<12288, F>(p, grid, stream);
    case 16384: return launch_parse_c<16384, F>(p, grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

// Host-side launch helper (same translation unit as the kernels).
cudaError_t launch_parse(const LaunchParams& p, int chunk_bytes, int grid, cudaStream_t stream,
                         bool f32) {
  return f32 ? launch_parse_f<F32>(p, chunk_bytes, grid, stream)
             : launch_parse_f<F64>(p, chunk_bytes, grid, stream);
}

template <int C, class F>
static cudaError_t occupancy_c(int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(parse_kernel<C, F, 0>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Layout<C>::TOTAL);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, parse_kernel<C, F, 0>, NT,
                                                       Layout<C>::TOTAL);
}

template <class F>
static cudaError_t occupancy_f(int chunk_bytes, int* blocks_per_sm) {
  switch (chunk_bytes) {
    case 4096: return occupancy_c<4096, F>(blocks_per_sm);
    case 8192: return occupancy_c<8192, F>(blocks_per_sm);
    case 12288: return occupancy_c<12288, F>(blocks_per_sm);
    case 16384: return occupancy_c<16384, F>(blocks_per_sm);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t parse_occupancy(int chunk_bytes, int* blocks_per_sm, bool f32) {
  return f32 ? occupancy_f<F32>(chunk_bytes, blocks_per_sm)
             : occupancy_f<F64>(chunk_bytes, blocks_per_sm);
}

}  // namespace fp
