/* oracle_sanitize.c -- drives the oracle (oracle/oracle.c, linked in) over
 * standard input, for a build with sanitizers: the whole buffer in both
 * formats under the three grammars on four threads (',' and '\n' as
 * separators), then every field alone from an exact-size copy, so that any
 * read past a field or a buffer is caught.  Prints "ok <fields>". */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

int oracle_parse_field_ex(const char *s, size_t n, int f32, int grammar, uint64_t *out_bits,
                          uint8_t *status);
uint64_t oracle_count_fields(const char *text, size_t len, char delim);
int oracle_parse_buffer_ex(const char *text, size_t len, char delim, int f32, int grammar,
                           void *out_bits, uint8_t *out_status, uint64_t cap, uint64_t *count,
                           int nthreads);

int main(int argc, char **argv) {
  const int buffer_only = argc > 1 && strcmp(argv[1], "buffer") == 0;
  size_t cap = 1 << 20, len = 0, got;
  char *in = malloc(cap);
  while (in && (got = fread(in + len, 1, cap - len, stdin)) > 0) {
    len += got;
    if (len == cap) {
      cap *= 2;
      in = realloc(in, cap);
    }
  }
  if (!in) return 2;
  char *text = malloc(len ? len : 1); /* exact size: a read past the end is caught */
  if (!text) return 2;
  memcpy(text, in, len);
  free(in);
  const uint64_t n = oracle_count_fields(text, len, ',');
  for (int f32 = 0; f32 < 2; f32++)
    for (int grammar = 0; grammar < 3; grammar++) {
      uint64_t *bits = malloc(8 * (n ? n : 1));
      uint8_t *st = malloc(n ? n : 1);
      uint64_t cnt = 0;
      if (!bits || !st) return 2;
      if (oracle_parse_buffer_ex(text, len, ',', f32, grammar, bits, st, n, &cnt, 4) || cnt != n) {
        printf("FAIL buffer f32=%d grammar=%d\n", f32, grammar);
        return 1;
      }
      free(bits);
      free(st);
    }
  size_t p = 0;
  while (!buffer_only && p <= len) {
    size_t q = p;
    while (q < len && text[q] != '\n' && text[q] != ',') q++;
    char *f = malloc(q > p ? q - p : 1);
    if (!f) return 2;
    memcpy(f, text + p, q - p);
    for (int k = 0; k < 6; k++) {
      uint64_t b;
      uint8_t s;
      oracle_parse_field_ex(f, q - p, k & 1, k >> 1, &b, &s);
    }
    free(f);
    p = q + 1;
  }
  free(text);
  printf("ok %llu\n", (unsigned long long)n);
  return 0;
}
