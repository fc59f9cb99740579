// fp_internal.h -- entry points that the library's own host runtime (the
// request server) uses beside the C ABI.  Not exported.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/fpparse.h"

namespace fp {

// fp_parse_f64_batch with explicit output ranges: buffer b writes entries
// [out_base[b], out_base[b] + out_cap[b]) of out_f64 / out_status (ranges
// of different buffers must not overlap) and its field count to
// out_counts[b].  err_out (optional, a device address, e.g. of pinned host
// memory) receives the stream's error word at the end of the call.
fp_err_t parse_batch_ranges(const char* const* texts, const size_t* lens, uint32_t nbuf,
                            char delim, double* out_f64, uint8_t* out_status,
                            const uint64_t* out_base, const uint64_t* out_cap,
                            uint64_t* out_counts, cudaStream_t stream,
                            unsigned int* err_out = nullptr);

// The pipelined host parse's segments: at most this many per text.
constexpr int PIPE_MAX_SEGS = 64;
// Texts of at least this many bytes in pinned memory are parsed in segments
// whose copies in, parses and copies out overlap.
constexpr size_t PIPE_MIN_BYTES = 32u << 20;

// Segment starts of a host text, cuts[0] = 0 < cuts[1] < ... < cuts[K] = len
// (returns K <= PIPE_MAX_SEGS; cuts has room for PIPE_MAX_SEGS + 1): each
// cut follows a separator ('\n' or delim), so a segment's fields are
// exactly the text's fields in that range.
int plan_host_segments(const char* host_text, size_t len, char delim, size_t* cuts);

// Grow the scratch of (current device, stream) now, so that later calls of
// up to `chunks` chunks and `nbuf` buffers allocate nothing.
fp_err_t reserve_stream_scratch(cudaStream_t stream, unsigned long long chunks, uint32_t nbuf);

// Synchronise `stream` and free its scratch (before the stream is destroyed).
fp_err_t release_stream_scratch(cudaStream_t stream);

// Device address of the error word of (current device, stream)'s scratch.
fp_err_t stream_error_word(cudaStream_t stream, unsigned int** word);

}  // namespace fp
