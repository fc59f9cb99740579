/*
 * fpparse_bench.h -- measurement support of libfpparse (not part of the
 * parsing API): replay a trace of timed parse requests, from native threads,
 * through the request server or through the plain per-request entry point,
 * so that the client keeps to the arrival schedule and the measured latency
 * is the server's (a client written in an interpreter falls behind the
 * schedule at tens of thousands of requests a second).
 */
#ifndef FPPARSE_BENCH_H
#define FPPARSE_BENCH_H

#include "fpparse.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One request body: host text and its host result arrays (pinned memory
 * copies fastest), as for fp_server_submit.  Requests of the same body may
 * be in flight together: they write the same values into the same arrays. */
typedef struct {
    const char *host_text;
    size_t len;
    double *host_f64;
    uint8_t *host_status;
    size_t out_cap;
} fp_replay_body_t;

/*
 * fp_replay_server -- request i (body bodies[order[i]]) is submitted to
 * `server` at t0 + arrival_ns[i], t0 being the steady-clock time of the call
 * plus lead_ns; a second thread waits for the requests in order.  Per request
 * out_ns[4 i .. 4 i + 3] = its arrival time, submission time, launch time and
 * completion time (steady-clock nanoseconds, the last two as the server
 * recorded them); n_bodies bounds order[].  Returns FP_OK, the first request's
 * error, or FP_ERR_ARG.  Synchronous.
 */
FP_API fp_err_t fp_replay_server(fp_server *server, const fp_replay_body_t *bodies,
                                 uint32_t n_bodies, const uint32_t *order,
                                 const int64_t *arrival_ns, size_t n, int64_t lead_ns,
                                 int64_t *out_ns);

/*
 * fp_replay_plain -- the same trace through fp_parse_f64_host on `stream`,
 * one request at a time: request i starts at its arrival time or when the
 * previous one has finished, whichever is later.  out_ns[2 i] = its arrival
 * time, out_ns[2 i + 1] = its completion time (steady clock).  Returns FP_OK,
 * the first request's error, or FP_ERR_ARG.  Synchronous.
 */
FP_API fp_err_t fp_replay_plain(const fp_replay_body_t *bodies, uint32_t n_bodies,
                                const uint32_t *order, const int64_t *arrival_ns, size_t n,
                                int64_t lead_ns, char delim, struct CUstream_st *stream,
                                int64_t *out_ns);

#ifdef __cplusplus
}
#endif
#endif /* FPPARSE_BENCH_H */
