/* c_client.c -- a plain C program linked against libfpparse.so: the calls
 * that need no GPU (sizes, error strings, argument checks) behave as the
 * header states.  Prints "ok" or the first failure. */
#include <stdio.h>
#include <string.h>

#include "fpparse.h"

#define CHECK(c)                                  \
  do {                                            \
    if (!(c)) {                                   \
      printf("FAIL line %d: %s\n", __LINE__, #c); \
      return 1;                                   \
    }                                             \
  } while (0)

int main(void) {
  uint64_t count = 0;
  double v[4];
  uint8_t st[4];
  CHECK(fp_max_fields(0) == 0 && fp_max_fields(12345) == 12345);
  CHECK(strcmp(fp_strerror(FP_OK), "ok") == 0);
  CHECK(strlen(fp_strerror(FP_ERR_ARG)) > 0 && strlen(fp_strerror((fp_err_t)99)) > 0);
  /* argument errors come back before anything is queued */
  CHECK(fp_parse_f64(NULL, 4, '\n', v, st, &count, NULL) == FP_ERR_ARG);
  CHECK(fp_parse_f64((const char *)v, 4, '\n', NULL, st, &count, NULL) == FP_ERR_ARG);
  CHECK(fp_parse_f64((const char *)v, 4, '\n', v, st, NULL, NULL) == FP_ERR_ARG);
  CHECK(fp_parse_f32(NULL, 4, '\n', (float *)v, st, &count, NULL) == FP_ERR_ARG);
  CHECK(fp_parse_f64_host(NULL, 4, '\n', v, st, &count, NULL) == FP_ERR_ARG);
  CHECK(fp_parse_f64_host("1\n", 2, '\n', v, st, NULL, NULL) == FP_ERR_ARG);
  fp_options_t opt;
  memset(&opt, 0, sizeof(opt));
  opt.delim = '\n';
  opt.grammar = 7; /* no such grammar */
  CHECK(fp_parse_ex((const char *)v, 4, &opt, v, st, &count, NULL) == FP_ERR_ARG);
  CHECK(fp_parse_ex((const char *)v, 4, NULL, v, st, &count, NULL) == FP_ERR_ARG);
  fp_config_t cfg, bad;
  CHECK(fp_get_config(&cfg) == FP_OK);
  bad = cfg;
  bad.chunk_bytes = 5000;
  CHECK(fp_set_config(&bad) == FP_ERR_ARG);
  bad = cfg;
  bad.ctas_per_sm = 9;
  CHECK(fp_set_config(&bad) == FP_ERR_ARG);
  CHECK(fp_set_config(&cfg) == FP_OK);
  CHECK(fp_get_stats(NULL, 0, NULL) == FP_ERR_ARG);
  CHECK(fp_batch_plan_launch(NULL, NULL) == FP_ERR_ARG);
  CHECK(fp_batch_plan_gather(NULL, NULL, NULL, NULL, NULL) == FP_ERR_ARG);
  CHECK(fp_server_create(NULL, NULL) == FP_ERR_ARG);
  CHECK(fp_server_destroy(NULL) == FP_OK);
  printf("ok\n");
  return 0;
}
