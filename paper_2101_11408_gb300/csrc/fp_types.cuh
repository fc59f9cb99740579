// fp_types.cuh -- structures shared by the kernels and the host launcher.
#pragma once
#include <cstdint>

namespace fp {

// One text buffer of a launch.  Offsets are in "aligned coordinates": the
// buffer's bytes occupy [o, o + len) relative to base, base being the text
// pointer rounded down to 16 bytes.
struct BufDesc {
  const uint8_t* base;
  unsigned long long o;
  unsigned long long len;
  unsigned long long chunk0;   // first global chunk of this buffer
  unsigned long long nchunks;  // chunks of this buffer (>= 1)
  unsigned long long out_base; // output index of field 0
  unsigned long long out_cap;  // output slots owned by this buffer
  unsigned long long* out_count;
};

// Per-stream control block.  The parse kernel's last block resets `ticket`
// and `done_parse`; the fallback kernel's last block resets the queue
// counters, so every call starts from zeros.
struct Ctl {
  unsigned long long ticket;     // next global chunk to hand out
  unsigned long long qcount;     // fallback queue appends (may exceed capacity)
  unsigned long long ovf_count;  // chunks whose pending fields overflowed the queue
  unsigned int done_parse;
  unsigned int done_fallback;
  unsigned int error;            // first device-side error of the stream (sticky)
  unsigned int pad0;
  unsigned long long stats[16];
};

struct LaunchParams {
  const BufDesc* descs;  // device array of nbuf descriptors (nbuf > 1)
  BufDesc one;           // the descriptor when nbuf == 1
  unsigned int nbuf;
  unsigned int delim;
  unsigned long long total_chunks;
  unsigned long long* out_bits;  // the caller's double (or float) array, as bit patterns
  uint8_t* out_status;
  Ctl* ctl;
  unsigned long long* chunk_status;  // look-back words, one per chunk
  unsigned int epoch;                // tag of this call's look-back words
  unsigned int pad0;
  unsigned long long* queue;         // fallback queue: output indices
  unsigned long long qcap;
  unsigned long long* ovf;           // overflow chunk list: (loc, out_base | n) pairs
  unsigned long long ovf_cap;
  // where a pending field's text location is kept until the fallback kernel
  // decides it, indexed like the outputs: out_bits itself for binary64
  // (the 8-byte slot holds it), a side array for binary32
  unsigned long long* loc;
  unsigned int grammar;     // GRAMMAR_* (fp_device.cuh); read by the slow paths
  unsigned int columns;     // K >= 2: column-major results (field i -> column i mod K)
  unsigned long long rows_cap;   // entries per column
  unsigned long long col_magic;  // ceil(2^64 / K): i div K = mulhi(i, magic) for i < 2^40
  // How long a device wait (look-back word, staging barrier) may spin before
  // it gives up with DERR_TIMEOUT; 0 means the default, WAIT_NS_DEFAULT.
  unsigned long long wait_ns;
  // Optional (null: unused), e.g. pinned host memory through its device
  // address: at the end of the call the fallback kernel's last block stores
  // the stream's error word (Ctl::error) here, so that the host learns the
  // call's outcome without a copy of its own.
  unsigned int* err_out;
  // Optional (null: unused), pinned host memory through its device address:
  // the fallback kernel stores how many fields the call queued for it (queue
  // appends plus overflow chunks; 0 when none), so that the host can tell
  // whether the stream's calls have fallback work.
  unsigned long long* pending_out;
};

constexpr unsigned long long WAIT_NS_DEFAULT = 2000000000ull;  // 2 s

// Look-back word: epoch (24 bits) | flag (2 bits) | value (38 bits).
constexpr int LB_VALUE_BITS = 38;
constexpr unsigned long long LB_VALUE_MASK = (1ull << LB_VALUE_BITS) - 1;
constexpr unsigned long long LB_FLAG_AGG = 1;
constexpr unsigned long long LB_FLAG_INC = 2;
constexpr unsigned int LB_EPOCH_MAX = (1u << 24) - 1;

// Location word stored in the output slot of a pending field:
// descriptor index (24 bits) << 40 | byte offset within the buffer (40 bits).
constexpr int LOC_OFF_BITS = 40;
constexpr unsigned long long LOC_OFF_MASK = (1ull << LOC_OFF_BITS) - 1;

}  // namespace fp
