/*
 * Open-loop load generator for the serving loop (sindi_server_*), used by
 * bench.py. Measurement infrastructure only: the library never calls it.
 *
 * Requests arrive at the times of a Poisson process of the offered rate
 * (exponential gaps, drawn up front). The calling thread submits each
 * request at its scheduled time (spinning on a monotonic clock); a second
 * thread polls the tickets in order. A request's latency runs from its
 * SCHEDULED arrival, not from the moment it was actually submitted, so a
 * submitter that falls behind the schedule (or a server that makes it wait)
 * shows up in the latency instead of being hidden (no coordinated
 * omission): latency = (submit time - scheduled time) + the server's own
 * submit-to-results time.
 *
 * The sindi_server_submit / sindi_server_poll entry points are passed in as
 * function pointers taken from the library the caller already loaded, so
 * this file links against nothing but libc and pthreads.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

typedef int (*submit_fn)(void* server, const int32_t* idx, const float* val, int32_t nnz, uint64_t* ticket);
typedef int (*poll_fn)(void* server, uint64_t ticket, int32_t wait_ms, uint32_t* ids, float* scores,
                       double* latency_ms);

typedef struct {
    double offered_qps;        /* the schedule's rate                                        */
    double achieved_qps;       /* completed requests / (last completion - first arrival)     */
    double seconds;            /* length of the schedule                                     */
    int64_t requests;
    int64_t failed;            /* requests whose submit or poll returned an error            */
    double p50_ms, p99_ms, max_ms, mean_ms;      /* scheduled arrival -> results on the host  */
    double server_p50_ms, server_p99_ms;         /* submit -> results (the server's figure)   */
    double lag_p99_ms, lag_max_ms;               /* submit time - scheduled time              */
} sindi_load_result;

static double now_s(void) {
    struct timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return (double)t.tv_sec + 1e-9 * (double)t.tv_nsec;
}

/* SplitMix64 (Steele, Lea, Flood 2014), for the arrival gaps. */
static uint64_t splitmix64(uint64_t* s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct {
    void* server;
    poll_fn poll;
    int64_t n;
    uint32_t k;
    uint64_t* tickets;
    volatile int* posted;      /* 1 when tickets[i] is valid, 2 when its submit failed */
    double* server_ms;
    double* done_s;
    int* ok;
} poller_args;

static void* poller(void* p) {
    poller_args* a = (poller_args*)p;
    uint32_t* ids = (uint32_t*)malloc(sizeof(uint32_t) * a->k);
    float* sc = (float*)malloc(sizeof(float) * a->k);
    for (int64_t i = 0; i < a->n; i++) {
        int st;
        while ((st = __atomic_load_n(&a->posted[i], __ATOMIC_ACQUIRE)) == 0) {
        }
        if (st != 1) {
            a->ok[i] = 0;
            continue;
        }
        double lat = 0.0;
        const int rc = a->poll(a->server, a->tickets[i], -1, ids, sc, &lat);
        a->done_s[i] = now_s();
        a->server_ms[i] = lat;
        a->ok[i] = rc == 0;
    }
    free(ids);
    free(sc);
    return NULL;
}

static int cmp_double(const void* x, const void* y) {
    const double a = *(const double*)x, b = *(const double*)y;
    return (a > b) - (a < b);
}

static double pct(const double* sorted, int64_t n, double q) {
    if (n <= 0) return 0.0;
    int64_t i = (int64_t)ceil(q * (double)n) - 1;
    if (i < 0) i = 0;
    if (i >= n) i = n - 1;
    return sorted[i];
}

/*
 * Runs one open-loop schedule of `seconds` at `offered_qps` over the query rows
 * (CSR qp/qx/qv, nrows rows, taken in turn) and fills *out. Returns 0, or -1
 * for bad arguments or an allocation failure (nothing submitted).
 */
int sindi_load_open_loop(void* server, void* submit_ptr, void* poll_ptr, const int64_t* qp, const int32_t* qx,
                         const float* qv, int64_t nrows, uint32_t k, double offered_qps, double seconds,
                         uint64_t seed, sindi_load_result* out) {
    if (!server || !submit_ptr || !poll_ptr || !qp || nrows <= 0 || k == 0 || !(offered_qps > 0.0) ||
        !(seconds > 0.0) || !out)
        return -1;
    submit_fn submit = (submit_fn)submit_ptr;
    const int64_t n = (int64_t)ceil(offered_qps * seconds);
    double* sched = (double*)malloc(sizeof(double) * n);
    double* lag = (double*)malloc(sizeof(double) * n);
    double* server_ms = (double*)calloc(n, sizeof(double));
    double* done_s = (double*)calloc(n, sizeof(double));
    double* lat = (double*)malloc(sizeof(double) * n);
    uint64_t* tickets = (uint64_t*)calloc(n, sizeof(uint64_t));
    int* posted = (int*)calloc(n, sizeof(int));
    int* ok = (int*)calloc(n, sizeof(int));
    if (!sched || !lag || !server_ms || !done_s || !lat || !tickets || !posted || !ok) {
        free(sched), free(lag), free(server_ms), free(done_s), free(lat), free(tickets), free(posted), free(ok);
        return -1;
    }
    uint64_t s = seed;
    double t = 0.0;
    for (int64_t i = 0; i < n; i++) {
        /* exponential gap: -ln(U) / rate, U uniform in (0, 1] from the top 53 bits */
        const double u = ((double)(splitmix64(&s) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
        t += -log(u) / offered_qps;
        sched[i] = t;
    }
    poller_args pa = {server, (poll_fn)poll_ptr, n, k, tickets, posted, server_ms, done_s, ok};
    pthread_t th;
    if (pthread_create(&th, NULL, poller, &pa) != 0) {
        free(sched), free(lag), free(server_ms), free(done_s), free(lat), free(tickets), free(posted), free(ok);
        return -1;
    }
    const double t0 = now_s();
    for (int64_t i = 0; i < n; i++) {
        const double due = t0 + sched[i];
        while (now_s() < due) {
        }
        const int64_t r = i % nrows;
        const int64_t b = qp[r], e = qp[r + 1];
        uint64_t ticket = 0;
        const double ts = now_s();
        const int rc = submit(server, qx + b, qv + b, (int32_t)(e - b), &ticket);
        lag[i] = 1e3 * (ts - due);
        tickets[i] = ticket;
        __atomic_store_n(&posted[i], rc == 0 ? 1 : 2, __ATOMIC_RELEASE);
    }
    pthread_join(th, NULL);
    int64_t good = 0, failed = 0;
    double last = t0, sum = 0.0;
    for (int64_t i = 0; i < n; i++) {
        if (!ok[i]) {
            failed++;
            continue;
        }
        lat[good] = lag[i] + server_ms[i];
        sum += lat[good];
        server_ms[good] = server_ms[i];
        if (done_s[i] > last) last = done_s[i];
        good++;
    }
    qsort(lat, good, sizeof(double), cmp_double);
    qsort(server_ms, good, sizeof(double), cmp_double);
    qsort(lag, n, sizeof(double), cmp_double);
    memset(out, 0, sizeof(*out));
    out->offered_qps = offered_qps;
    out->seconds = seconds;
    out->requests = n;
    out->failed = failed;
    out->achieved_qps = last > t0 ? (double)good / (last - t0) : 0.0;
    out->p50_ms = pct(lat, good, 0.50);
    out->p99_ms = pct(lat, good, 0.99);
    out->max_ms = good ? lat[good - 1] : 0.0;
    out->mean_ms = good ? sum / (double)good : 0.0;
    out->server_p50_ms = pct(server_ms, good, 0.50);
    out->server_p99_ms = pct(server_ms, good, 0.99);
    out->lag_p99_ms = pct(lag, n, 0.99);
    out->lag_max_ms = n ? lag[n - 1] : 0.0;
    free(sched), free(lag), free(server_ms), free(done_s), free(lat), free(tickets), free(posted), free(ok);
    return 0;
}
