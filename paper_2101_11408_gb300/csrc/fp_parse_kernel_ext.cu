// fp_parse_kernel_ext.cu -- the parse kernel's JSON, hexadecimal and
// column-major modes (fp_parse_ex), for 8 KiB and 16 KiB chunks; the kernel
// itself is in fp_parse_kernel.cuh.
#include "fp_launch.h"
#include "fp_parse_kernel.cuh"

namespace fp {

template <int C, class F, int MODE>
static cudaError_t launch_ext_c(const LaunchParams& p, int grid, cudaStream_t stream) {
  static bool attr_set = false;  // the attribute is per function; set it once
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(parse_kernel<C, F, MODE>,
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
  return cudaLaunchKernelEx(&cfg, parse_kernel<C, F, MODE>, p);
}

template <int C, class F>
static cudaError_t launch_ext_f(const LaunchParams& p, int grid, cudaStream_t stream, int mode) {
  switch (mode) {
    case MODE_JSON: return launch_ext_c<C, F, MODE_JSON>(p, grid, stream);
    case MODE_COLUMNS: return launch_ext_c<C, F, MODE_COLUMNS>(p, grid, stream);
    case MODE_JSON | MODE_COLUMNS: return launch_ext_c<C, F, MODE_JSON | MODE_COLUMNS>(p, grid, stream);
    case MODE_HEX: return launch_ext_c<C, F, MODE_HEX>(p, grid, stream);
    case MODE_HEX | MODE_COLUMNS: return launch_ext_c<C, F, MODE_HEX | MODE_COLUMNS>(p, grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_parse_ext(const LaunchParams& p, int chunk_bytes, int grid,
                             cudaStream_t stream, bool f32, int mode) {
  if (chunk_bytes == 8192)
    return f32 ? launch_ext_f<8192, F32>(p, grid, stream, mode)
               : launch_ext_f<8192, F64>(p, grid, stream, mode);
  if (chunk_bytes == 16384)
    return f32 ? launch_ext_f<16384, F32>(p, grid, stream, mode)
               : launch_ext_f<16384, F64>(p, grid, stream, mode);
  return cudaErrorInvalidValue;
}

template <int C, class F, int MODE>
static cudaError_t occupancy_ext_c(int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(parse_kernel<C, F, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Layout<C>::TOTAL);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, parse_kernel<C, F, MODE>,
                                                       NT, Layout<C>::TOTAL);
}

// The blocks per SM that every instance of one chunk size reaches (the
// persistent grid must be resident whole, whichever instance runs).
template <int C>
static cudaError_t occupancy_ext_all(int* blocks_per_sm) {
  int b[8], k = 0;
  cudaError_t e = cudaSuccess;
  for (int f32 = 0; f32 < 2 && e == cudaSuccess; f32++) {
    for (int m : {MODE_JSON, MODE_JSON | MODE_COLUMNS, MODE_HEX, MODE_HEX | MODE_COLUMNS}) {
      if (e != cudaSuccess) break;
      if (f32) {
        switch (m) {
          case MODE_JSON: e = occupancy_ext_c<C, F32, MODE_JSON>(&b[k]); break;
          case MODE_JSON | MODE_COLUMNS: e = occupancy_ext_c<C, F32, MODE_JSON | MODE_COLUMNS>(&b[k]); break;
          case MODE_HEX: e = occupancy_ext_c<C, F32, MODE_HEX>(&b[k]); break;
          default: e = occupancy_ext_c<C, F32, MODE_HEX | MODE_COLUMNS>(&b[k]); break;
        }
      } else {
        switch (m) {
          case MODE_JSON: e = occupancy_ext_c<C, F64, MODE_JSON>(&b[k]); break;
          case MODE_JSON | MODE_COLUMNS: e = occupancy_ext_c<C, F64, MODE_JSON | MODE_COLUMNS>(&b[k]); break;
          case MODE_HEX: e = occupancy_ext_c<C, F64, MODE_HEX>(&b[k]); break;
          default: e = occupancy_ext_c<C, F64, MODE_HEX | MODE_COLUMNS>(&b[k]); break;
        }
      }
      k++;
    }
  }
  if (e != cudaSuccess) return e;
  int mn = b[0];
  for (int i = 1; i < k; i++) mn = b[i] < mn ? b[i] : mn;
  *blocks_per_sm = mn;
  return cudaSuccess;
}

cudaError_t parse_occupancy_ext(int chunk_bytes, int* blocks_per_sm) {
  if (chunk_bytes == 8192) return occupancy_ext_all<8192>(blocks_per_sm);
  if (chunk_bytes == 16384) return occupancy_ext_all<16384>(blocks_per_sm);
  return cudaErrorInvalidValue;
}

}  // namespace fp
