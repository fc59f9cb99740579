// swar_check.cpp -- the word-wide byte tests of the device header, built for
// the host, against byte-by-byte definitions: the zero-byte, separator and
// non-digit flags are exact in every byte; two words of flags become the
// right 8-bit mask; four ASCII digits give their value; the funnel shift
// matches its definition; the window tokenizer's tables move and keep the
// bytes their definitions say.  Prints "ok" or the first failure.
#include <cstdio>
#include <cstdint>
#include <random>

#include "fp_device.cuh"

using namespace fp;

namespace {

uint8_t byte_of(uint32_t w, int i) { return (uint8_t)(w >> (8 * i)); }

bool is_dig(uint8_t c) { return c >= '0' && c <= '9'; }

int fail(const char* what, uint32_t a, uint32_t b = 0) {
  std::printf("FAIL %s %08x %08x\n", what, a, b);
  return 1;
}

}  // namespace

int main() {
  std::mt19937_64 rng(0x2101114081ull);
  // a byte drawn to hit digits, their neighbours and the separators often
  const uint8_t special[] = {'0', '1', '5', '9', '/', ':', '.', 'e', 'E', '+', '-', ' ', '\n',
                             ',', 0, 0x7F, 0x80, 0xFF, 0x2F, 0x3A, 0xB0, 0xB9};
  auto rand_byte = [&]() -> uint8_t {
    const uint64_t r = rng();
    return (r & 1) ? special[(r >> 1) % sizeof(special)] : (uint8_t)(r >> 8);
  };
  auto rand_word = [&]() -> uint32_t {
    uint32_t w = 0;
    for (int i = 0; i < 4; i++) w |= (uint32_t)rand_byte() << (8 * i);
    return w;
  };
  for (int it = 0; it < 4000000; it++) {
    const uint32_t w = rand_word();
    // zero_bytes: 0x80 exactly in the zero bytes
    const uint32_t z = zero_bytes(w);
    for (int i = 0; i < 4; i++)
      if ((byte_of(z, i) == 0x80) != (byte_of(w, i) == 0) || (byte_of(z, i) & 0x7F))
        return fail("zero_bytes", w, z);
    // sep_flags_one / sep_flags_two: 0x80 exactly in the bytes equal to a
    // separator ('\n', and a second one below 0x80)
    const uint8_t sep2 = (uint8_t)(rng() % 0x80);
    const uint32_t p1 = 0x0A0A0A0Au, p2 = sep2 * 0x01010101u;
    const uint32_t s1 = sep_flags_one(w, p1), s2 = sep_flags_two(w, p1, p2);
    for (int i = 0; i < 4; i++) {
      const uint8_t c = byte_of(w, i);
      if ((byte_of(s1, i) == 0x80) != (c == '\n') || (byte_of(s1, i) & 0x7F))
        return fail("sep_flags_one", w, s1);
      if ((byte_of(s2, i) == 0x80) != (c == '\n' || c == sep2) || (byte_of(s2, i) & 0x7F))
        return fail("sep_flags_two", w, p2);
    }
    // nondigit_exact: 0x80 exactly in the bytes that are not '0'..'9'
    const uint32_t nd = nondigit_exact(w);
    for (int i = 0; i < 4; i++)
      if ((byte_of(nd, i) == 0x80) == is_dig(byte_of(w, i)) || (byte_of(nd, i) & 0x7F))
        return fail("nondigit_exact", w, nd);
    // the funnel shift
    const uint32_t w2 = rand_word();
    const uint32_t sh = (uint32_t)(rng() % 32);
    const uint64_t cat = ((uint64_t)w2 << 32) | w;
    if (fshr(w, w2, sh) != (uint32_t)(cat >> sh)) return fail("fshr", w, sh);
  }
  // the window tables: every point position moves exactly the bytes at or
  // before it one place toward the end; every mask keeps exactly its bytes
  {
    WindowTables wt;
    for (int i = 0; i < WINDOW_TABLE_WORDS; i++)
      reinterpret_cast<uint32_t*>(&wt)[i] = window_table_word(i);
    uint8_t win[24];
    for (int i = 0; i < 24; i++) win[i] = (uint8_t)('A' + i);
    for (int d = 0; d <= 24; d++) {
      uint32_t prev = 0x30303030u;
      for (int j = 0; j < 6; j++) {
        uint32_t xj = 0;
        for (int b = 0; b < 4; b++) xj |= (uint32_t)win[4 * j + b] << (8 * b);
        const uint32_t r = byte_perm(prev, xj, wt.sel[j][d]);
        prev = xj;
        for (int b = 0; b < 4; b++) {
          const int p = 4 * j + b;
          const uint8_t want = (d < 24 && p <= d) ? (p == 0 ? '0' : win[p - 1]) : win[p];
          if (byte_of(r, b) != want) return fail("window sel", (uint32_t)d, (uint32_t)p);
        }
      }
    }
    for (int l = 0; l <= 24; l++)
      for (int p = 0; p < 24; p++)
        if ((byte_of(wt.keep_from[p / 4][l], p % 4) == 0xFF) != (p >= l) ||
            (byte_of(wt.keep_from[p / 4][l], p % 4) != 0 && byte_of(wt.keep_from[p / 4][l], p % 4) != 0xFF))
          return fail("window keep_from", (uint32_t)l, (uint32_t)p);
    for (int m = 16; m <= 24; m++)
      for (int p = 16; p < 24; p++) {
        const uint8_t k = byte_of(wt.keep_below[(p - 16) / 4][m - 16], p % 4);
        if ((k == 0xFF) != (p < m) || (k != 0 && k != 0xFF))
          return fail("window keep_below", (uint32_t)m, (uint32_t)p);
      }
  }
  // flag_pair: every pattern of flags in two words
  for (uint32_t m = 0; m < 256; m++) {
    uint32_t w0 = 0, w1 = 0;
    for (int b = 0; b < 4; b++) {
      if (m & (1u << b)) w0 |= 0x80u << (8 * b);
      if (m & (1u << (4 + b))) w1 |= 0x80u << (8 * b);
    }
    if (flag_pair(w0, w1) != 128u * m) return fail("flag_pair", w0, w1);
  }
  // dig4: all four-digit strings, first byte most significant
  for (uint32_t v = 0; v < 10000; v++) {
    const uint32_t x = (uint32_t)('0' + v / 1000) | (uint32_t)('0' + v / 100 % 10) << 8 |
                       (uint32_t)('0' + v / 10 % 10) << 16 | (uint32_t)('0' + v % 10) << 24;
    if (dig4(x) != v) return fail("dig4", x, v);
  }
  std::printf("ok\n");
  return 0;
}
