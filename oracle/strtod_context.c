/*
 * strtod_context.c -- the C library's strtod over a delimited buffer, split
 * across threads: a timing CONTEXT for the CPU baseline (the paper compares
 * its method with the C library's conversion), used only by bench.py.
 *
 * Not the oracle and not a checker: nothing is compared with these results
 * (each thread writes its values from an upper bound of its first field
 * index, so they are not in field order).  Fields are separated by '\n' or
 * the delimiter; every field is converted, the trailing empty field is not.
 */
#define _POSIX_C_SOURCE 200809L
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

typedef struct {
  const char *text;
  size_t begin, end; /* byte range; begin is a field start */
  char delim;
  double *out;       /* room for (end - begin) / 2 + 1 values */
  uint64_t count;
} job_t;

static void *run(void *arg) {
  job_t *j = (job_t *)arg;
  const char *s = j->text;
  size_t p = j->begin;
  uint64_t n = 0;
  while (p < j->end) {
    size_t e = p;
    while (e < j->end && s[e] != '\n' && s[e] != j->delim) e++;
    char *stop;
    j->out[n++] = strtod(s + p, &stop); /* stops at the separator (or the NUL) */
    p = e + 1;
  }
  j->count = n;
  return NULL;
}

/* Convert every field of text[0, len) with strtod on nthreads threads.
 * Returns 0 and the field count and the seconds spent converting (the copy
 * into a NUL-terminated buffer excluded), or -1 when memory runs out. */
int context_strtod_buffer(const char *text, size_t len, char delim, int nthreads,
                          uint64_t *count, double *seconds) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  char *buf = malloc(len + 1);
  double *out = malloc(sizeof(double) * (len / 2 + (size_t)nthreads + 1));
  job_t *jobs = calloc((size_t)nthreads, sizeof(job_t));
  pthread_t *th = calloc((size_t)nthreads, sizeof(pthread_t));
  if (!buf || !out || !jobs || !th) {
    free(buf);
    free(out);
    free(jobs);
    free(th);
    return -1;
  }
  memcpy(buf, text, len);
  buf[len] = '\0';
  /* range boundaries just after a separator */
  size_t prev = 0, out_off = 0;
  for (int t = 0; t < nthreads; t++) {
    size_t b = (t == nthreads - 1) ? len : len / (size_t)nthreads * (size_t)(t + 1);
    if (b < prev) b = prev;
    while (b > 0 && b < len && buf[b - 1] != '\n' && buf[b - 1] != delim) b++;
    jobs[t].text = buf;
    jobs[t].begin = prev;
    jobs[t].end = b;
    jobs[t].delim = delim;
    jobs[t].out = out + out_off;
    out_off += (b - prev) / 2 + 1;
    prev = b;
  }
  struct timespec t0, t1;
  clock_gettime(CLOCK_MONOTONIC, &t0);
  int started = 0;
  for (int t = 0; t < nthreads; t++, started++)
    if (pthread_create(&th[t], NULL, run, &jobs[t]) != 0) break;
  for (int t = started; t < nthreads; t++) run(&jobs[t]); /* threads refused: run here */
  for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
  clock_gettime(CLOCK_MONOTONIC, &t1);
  uint64_t n = 0;
  for (int t = 0; t < nthreads; t++) n += jobs[t].count;
  *count = n;
  *seconds = (double)(t1.tv_sec - t0.tv_sec) + 1e-9 * (double)(t1.tv_nsec - t0.tv_nsec);
  free(buf);
  free(out);
  free(jobs);
  free(th);
  return 0;
}
