// hot_path_check.cpp -- the parse kernel's per-field steps, built for the
// host from the device header (its functions are host-callable) and run on
// every '\n'-separated field of standard input: the window tokenizer of
// Section 4 on a padded tile (with its lookup tables as the kernel builds
// them), Algorithm 1 (Section 5) on its (w, q), in the hexadecimal grammar
// the hexadecimal window tokenizer for fields with an "0x" (as the kernel's
// hexadecimal mode does), and
// the general tokenizer with the 19-digit check of Section 11 for the fields
// the first one declines; fields both leave undecided are printed as "P"
// (the fallback kernel's).  One line per field: "<bits hex> <status>" or
// "P".  The test compares the decided ones with the oracle.  The number of
// fields the hexadecimal window decided goes to standard error.
//
// usage: hot_path_check <64|32> <grammar 0|1|2> < text
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "fp_device.cuh"

namespace {

constexpr int LEAD = 32;  // tile bytes before the field (parse_window reads up to 28)

fp::WindowTables g_wt;
long g_hex_window = 0;

template <class F>
void check_field(const uint8_t* field, int n, uint32_t grammar, const fp::Pow5& tab) {
  using namespace fp;
  alignas(16) uint8_t tile[LEAD + LMAX + 32];
  std::memset(tile, 0, sizeof(tile));
  if (n > LMAX) {  // the kernel hands longer fields to the fallback kernel
    std::printf("P\n");
    return;
  }
  std::memcpy(tile + LEAD, field, (size_t)n);
  tile[LEAD + n] = '\n';
  const int s = LEAD, e = LEAD + n;
  if (grammar == GRAMMAR_HEX) {
    const uint32_t c0 = tile[s];
    const int s1 = s + ((c0 == '-') | (c0 == '+'));
    if ((tile[s1 + 1] | 0x20u) == 'x') {
      uint64_t hbits = 0;
      uint8_t hst = ST_GENERAL;
      if (parse_hex_window<F>(tile, g_wt, s, e, hbits, hst)) {
        g_hex_window++;
        std::printf("%016llx %u\n", (unsigned long long)hbits, (unsigned)hst);
        return;
      }
      const FieldResult g = parse_short_field<F>(tile + s, n, tab, grammar);
      if (g.status == ST_PENDING) std::printf("P\n");
      else std::printf("%016llx %u\n", (unsigned long long)g.bits, (unsigned)g.status);
      return;
    }
  }
  FastToken ft;
  ft.w = 0;
  ft.q = 0;
  ft.sign = 0;
  bool ok = parse_window(tile, g_wt, s, e, ft);
  if (grammar == GRAMMAR_JSON) ok = ok && json_ok_fast(tile, s, ft);
  const ElResult r = convert_wq<F>(ft.w ? ft.w : 1ull, ok ? ft.q : 0, tab, true);
  uint64_t sgn = ft.sign;
  if (F::MBITS != F64::MBITS) sgn = ft.sign ? F::SIGN : 0;
  uint64_t bits = ft.w ? (r.bits | sgn) : sgn;
  unsigned status = !ok ? (unsigned)ST_GENERAL : (ft.w ? (unsigned)r.status : (unsigned)ST_OK);
  if (status == ST_GENERAL) {
    const FieldResult g = parse_short_field<F>(tile + s, n, tab, grammar);
    if (g.status == ST_PENDING) {
      std::printf("P\n");
      return;
    }
    bits = g.bits;
    status = g.status;
  }
  std::printf("%016llx %u\n", (unsigned long long)bits, status);
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 3) {
    std::fprintf(stderr, "usage: %s <64|32> <grammar>\n", argv[0]);
    return 2;
  }
  const bool f32 = std::atoi(argv[1]) == 32;
  const uint32_t grammar = (uint32_t)std::atoi(argv[2]);
  // the table as the kernel holds it: dense high words, interleaved low words
  static const unsigned long long table[2 * FP_POW5_ENTRIES] = {FP_POW5_TABLE_VALUES};
  static uint64_t hi[FP_POW5_ENTRIES];
  for (int i = 0; i < FP_POW5_ENTRIES; i++) hi[i] = table[2 * i];
  const fp::Pow5 tab{hi, 1, reinterpret_cast<const uint64_t*>(table) + 1};
  for (int i = 0; i < fp::WINDOW_TABLE_WORDS; i++)
    reinterpret_cast<uint32_t*>(&g_wt)[i] = fp::window_table_word(i);
  std::string text;
  char buf[1 << 16];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), stdin)) > 0) text.append(buf, got);
  // fields: the pieces between '\n's; a text ending in '\n' has no empty
  // field after it
  size_t p = 0;
  while (p < text.size()) {
    size_t q = text.find('\n', p);
    if (q == std::string::npos) q = text.size();
    const uint8_t* f = reinterpret_cast<const uint8_t*>(text.data()) + p;
    const int n = (int)(q - p);
    if (f32) check_field<fp::F32>(f, n, grammar, tab);
    else check_field<fp::F64>(f, n, grammar, tab);
    p = q + 1;
  }
  std::fprintf(stderr, "hex_window %ld\n", g_hex_window);
  return 0;
}
