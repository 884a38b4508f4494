/*
 * cch.h -- C ABI of the GB300 (sm_103a) CudaChain planar convex hull.
 *
 * The library computes the convex hull of planar point sets with the method
 * of G. Mei, "CudaChain: A Practical GPU-accelerated 2D Convex Hull
 * Algorithm" (arXiv:1508.05488): the four extreme points and the
 * quadrilateral discard with region routing (Sec. 2.1 steps 1-3, Sec. 2.1.1),
 * the per-region sort (step 4, Table 1), the Sorting-based Preprocessing
 * Approach (step 5, Fig. 2), and the simple polygon's hull (steps 6-7) --
 * every step on the GPU; the paper's CPU stage (Melkman's algorithm) is
 * replaced by a device chain-hull stage.
 *
 * OUTPUT CONTRACT (all entry points): the vertices of the STRICT convex hull
 * -- no point that lies on a hull edge between two vertices, no repeated
 * point -- as int32 indices into the input, counter-clockwise, starting at
 * the lexicographically smallest point (smallest x, then smallest y).  Among
 * points with identical coordinates the smallest index is reported.
 * Degenerate inputs: n = 0 -> no vertex; all points identical -> the one
 * (smallest) index; all points collinear -> the two end points.
 *
 * INPUT CONTRACT: points are a contiguous row-major [n, 2] array of int32 or
 * float64 (x, y) pairs, aligned to 8 (int32) / 16 (float64) bytes.
 *   int32   any values; orientation is exact in 64/128-bit integers.
 *   float64 finite, and each coordinate either 0 or of magnitude in
 *           [2^-400, 2^400); orientation is exact (filtered, then expansion
 *           arithmetic).  -0.0 equals +0.0.  A NaN/Inf is reported as
 *           CCH_ERR_NONFINITE, another value outside the range as
 *           CCH_ERR_RANGE, in the output count (see below).
 *   n       0 <= n <= 2^30 points per set, at most 2^31 - 1 in total.
 *
 * STREAMS AND OWNERSHIP: entry points taking a `stream` are asynchronous on
 * that CUDA stream (a cudaStream_t passed as void*; NULL = legacy default
 * stream).  Device buffers belong to the caller and must stay valid until
 * the stream reaches the call.  The library keeps one scratch workspace per
 * stream (device memory, grown on demand, reused by later calls on that
 * stream); cch_release_workspace() frees it.  Calls on one stream are
 * serialised by the stream; calls on different streams use different
 * workspaces and may overlap on the device.
 *
 * ERRORS: the return value reports what the host can see before launching
 * (bad arguments, allocation or launch failure) as a negative CCH_ERR_*
 * code; nothing is launched then.  Errors found on the device (non-finite or
 * out-of-range coordinates, an exhausted bounded wait) are written as the
 * negative code into the set's output count instead of a hull size.
 */
#ifndef CCH_H_
#define CCH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum cch_dtype { CCH_I32 = 1, CCH_F64 = 2 };

enum cch_status {
  CCH_OK = 0,
  CCH_ERR_INVALID = -1,    /* bad argument (NULL pointer, n < 0, misaligned) */
  CCH_ERR_DTYPE = -2,      /* dtype is neither CCH_I32 nor CCH_F64 */
  CCH_ERR_NONFINITE = -3,  /* a float64 coordinate is NaN or Inf */
  CCH_ERR_RANGE = -4,      /* size or coordinate magnitude outside the contract */
  CCH_ERR_NOMEM = -5,      /* device or host allocation failed */
  CCH_ERR_CUDA = -6,       /* a CUDA runtime call failed */
  CCH_ERR_TIMEOUT = -7,    /* a bounded device-side wait ran out */
  CCH_ERR_BUSY = -8,       /* serving: the pending queue is full */
  CCH_ERR_NOTFOUND = -9    /* serving: unknown ticket */
};

/* Static description of a status code. */
const char *cch_status_string(int status);

/*
 * One hull (Sec. 2.1, steps 1-7).
 *   points     device pointer to [n, 2] int32 / float64 (see INPUT CONTRACT)
 *   n          number of points
 *   dtype      CCH_I32 or CCH_F64
 *   out_idx    device int32[max(n, 1)]: receives the h hull indices
 *   out_count  device int32[1]: receives h, or a negative CCH_ERR_* code
 *   stream     cudaStream_t
 * Returns CCH_OK once the work is enqueued.
 */
int cch_hull(const void *points, int64_t n, int dtype,
             int32_t *out_idx, int32_t *out_count, void *stream);

/*
 * Many independent hulls in one launch sequence: set s is
 * points[offsets[s] .. offsets[s+1]) (offsets: HOST int64[nsets + 1],
 * offsets[0] = 0, non-decreasing).  Its hull indices are local to the set and
 * are written to out_idx + offsets[s]; its count (or a negative code) to
 * out_counts[s].  out_idx: device int32[max(offsets[nsets], 1)];
 * out_counts: device int32[nsets].  Same method and output contract as
 * cch_hull per set.
 */
int cch_hull_batched(const void *points, const int64_t *offsets, int32_t nsets,
                     int dtype, int32_t *out_idx, int32_t *out_counts, void *stream);

/*
 * End-to-end convenience form of cch_hull on HOST buffers: copies the points
 * to the device (from pinned or pageable host memory), computes the hull and
 * copies the count and the indices back; returns when they are in host memory.
 *   points_host  host [n, 2] int32 / float64
 *   out_idx_host host int32[max(n, 1)]
 *   out_count    host int32: h or a negative code
 * Returns CCH_OK or a negative code (the device-side code is also returned).
 */
int cch_hull_host(const void *points_host, int64_t n, int dtype,
                  int32_t *out_idx_host, int32_t *out_count, void *stream);

/*
 * The hull of points given as two float32 coordinate arrays, the input form
 * of the paper's implementation (Fig. 6 takes the coordinates as two float
 * vectors x and y).  Round 1 (the extremes, the quadrilateral test, region
 * routing and the dominance prefilter) reads the two vectors directly,
 * 8 bytes a point; its survivors and every later stage carry the points
 * widened exactly to float64 (sign, rebiased exponent, significand shifted;
 * subnormals normalised), so the result is cch_hull's on the points
 * (double(x[i]), double(y[i])): the same indices, the same rules for
 * duplicates, collinear points and -0.0.
 *   x, y       device float[n] each, 4-byte aligned (any offset within a
 *              16-byte line); caller-owned, read only
 *   n          0 <= n <= 2^30
 *   out_idx    device int32[max(n, 1)]; out_count device int32 (h, or a
 *              negative code: CCH_ERR_NONFINITE for NaN / Inf)
 * Uses the per-stream workspace of cch_hull.  Asynchronous on `stream`;
 * host-detectable errors return before any launch.
 */
int cch_hull_f32soa(const float *x, const float *y, int64_t n, int32_t *out_idx,
                    int32_t *out_count, void *stream);

/*
 * Intermediate sets of one hull, for stage-by-stage checking.
 *   opts          bit 0: evaluate every float64 quadrilateral test exactly
 *                 (no FP32 filter); bit 1: keep every round-1 survivor (no
 *                 SPA-dominance prefilter, so r1_idx is exactly the paper's
 *                 R1..R4); bit 2: the paper's chunked GPU SPA (Sec. 2.2.2:
 *                 per region one block of 1024 threads, thread t checking
 *                 sorted points [t L, (t+1) L), L = ceil(m / 1024), with
 *                 Fig. 2's rule restarted at its chunk's first point) gives
 *                 spa_idx and its counts, on the paper's round-1 sets (bit 2
 *                 implies bit 1; the hull still comes from the sequential
 *                 rule, so out_idx is unchanged); bit 3: round 1 discards
 *                 the points strictly inside the octagon of the four
 *                 extremes and four diagonal extremes (Akl-Toussaint, the
 *                 paper's reference [17]; D_r, the point with the smallest
 *                 FP32 score X+Y, Y-X, -X-Y, X-Y of its coordinates' views,
 *                 ties to the smallest index, between E_r and E_{r+1} when
 *                 it lies strictly outside that quadrilateral edge), instead
 *                 of the quadrilateral alone; implies bit 1; other bits
 *                 must be 0
 *   r1_idx        device int32[max(n,1)]: round-1 survivors (Sec. 2.1.1),
 *                 region after region, index order within a region
 *   r1_region     device int32[max(n,1)]: their regions 1..4
 *   spa_idx       device int32[max(n,1)]: SPA survivors (Fig. 2) of R1..R4
 *                 in sorted (Table 1) order, region after region
 *   counts_host   host int64[16]: s1, records of R1..R4, survivors of R1..R4,
 *                 the device status (0 or a negative code), the number of
 *                 LSD radix passes the multi-block sort ran (0 when the set
 *                 took the shared-memory path; byte passes whose digit is the
 *                 same for every record are skipped), with bit 3 the indices
 *                 of D_1..D_4 (-1 where unused; otherwise -1), and 0
 *   out_idx, out_count   as for cch_hull
 * Synchronises the stream before returning.
 */
int cch_hull_stages(const void *points, int64_t n, int dtype, uint32_t opts,
                    int32_t *r1_idx, int32_t *r1_region, int32_t *spa_idx,
                    int64_t *counts_host, int32_t *out_idx, int32_t *out_count,
                    void *stream);

/*
 * Stage timing.  cch_profile(1) makes every later call record CUDA events on
 * its stream around eight stages: (0) the extremes pass a1, (1) the
 * dominance-table sample, (2) the classify pass a2, (3) the gather of the
 * survivors into region order, (4) sort and SPA of the shared-memory path,
 * (5) sort and SPA of the multi-block path, (6) chain hull and output,
 * (7) the stage extraction of cch_hull_stages (with opts bit 2: the paper's
 * chunked SPA).  cch_profile_read synchronises on the recorded events, writes
 * the summed milliseconds per stage to stage_ms[0 .. min(8, max_stages)), the
 * number of calls to *calls (if not NULL), forgets them, and returns the
 * number of stages (8).  cch_profile(0) stops recording.  cch_profile_stages(mask)
 * records only around the stages whose bit is set in mask (bit k: stage k;
 * the others read as 0), which keeps the events' own cost out of the rest
 * of the pipeline; mask 0 stops recording.
 */
int cch_profile(int enable);
int cch_profile_stages(uint32_t mask);
int cch_profile_read(double *stage_ms, int max_stages, int64_t *calls);

/* Number of CUDA kernels this library has launched since it was loaded. */
uint64_t cch_launch_count(void);

/*
 * Self-test of the device-side failure path: one kernel waits on a device
 * flag that nothing sets, with the same bounded wait every kernel of the
 * library uses, and must give up and report.  Writes to *status_dev (device
 * int32) the status the wait recorded -- CCH_ERR_TIMEOUT when the path works
 * -- asynchronously on `stream`.  The context stays usable afterwards.
 */
int cch_selftest_wait(int32_t *status_dev, void *stream);

/*
 * cch_hull without any device-memory allocation, for callers that cannot
 * call cudaMalloc: code running under a CUDA graph capture that forbids
 * allocation, real-time or embedded callers whose device footprint is fixed
 * at load time, or code running inside an allocator's own callback.  The
 * paper has no counterpart; this is a property of this library only.
 *
 * Arguments, output and errors are those of cch_hull, for at most 131072
 * points (larger n returns CCH_ERR_RANGE and launches nothing).  Scratch is a
 * fixed 12 MiB array in the library's device code, held by every GPU that
 * loads the library until the process exits, and shared by every call on
 * that GPU: it keeps the previous call's contents (each call clears what must
 * start at zero), and calls whose work can overlap on the GPU -- different
 * streams without ordering between them -- race and give wrong results.  The
 * first call on each device looks up the array's address and clears it; make
 * that first call before any stream capture.
 */
int cch_hull_noalloc(const void *points, int64_t n, int dtype,
                     int32_t *out_idx, int32_t *out_count, void *stream);

/* ------------------------------------------------------------- tuning --
 * Run-time choices of a call, none of which changes a result: the largest
 * region sorted in shared memory (above it the multi-block sort runs), the
 * sample behind the dominance prefilter (m = min(n, stair_max, max(stair_min,
 * n / stair_div))), the smallest a1 chunk, and a2's CTAs per SM.  A table
 * keyed by GPU (name, SM count), dtype, single set or batch, and size bucket
 * (floor(log2(points per set)), cch_tune_bucket) holds them; calls without
 * an entry use the defaults.  The table can be filled by hand, by
 * cch_autotune_batched, or from a JSON cache file. */
typedef struct cch_tune_params {
  int32_t small_max;     /* 1 .. 16384 */
  int32_t stair_div;     /* >= 1 */
  int32_t stair_min;     /* 1 .. stair_max */
  int32_t stair_max;     /* <= 2^24 */
  int32_t a1_len_min;    /* 4096 .. 2^26, a multiple of 1024 */
  int32_t cls_per_sm;    /* 1 or 2 */
} cch_tune_params;

/* Size bucket of a call of npts points in nsets sets. */
int cch_tune_bucket(int64_t npts, int32_t nsets);
/* Set / get the entry of (gpu, sms, dtype, batched 0/1, bucket); gpu NULL
 * means the current device (sms ignored).  Set returns CCH_ERR_INVALID for
 * values outside the ranges above.  Get fills *p with the entry, or with the
 * defaults and returns CCH_ERR_NOTFOUND. */
int cch_tune_set(const char *gpu, int32_t sms, int32_t dtype, int32_t batched, int32_t bucket,
                 const cch_tune_params *p);
int cch_tune_get(const char *gpu, int32_t sms, int32_t dtype, int32_t batched, int32_t bucket,
                 cch_tune_params *p);
/* Forget every entry. */
int cch_tune_clear(void);
/* Write the table to a JSON file; merge a file written by cch_tune_save into
 * it (the whole file is checked first: CCH_ERR_INVALID leaves the table
 * unchanged, CCH_ERR_NOTFOUND if the file cannot be opened). */
int cch_tune_save(const char *path);
int cch_tune_load(const char *path);
/* Measure the choices on this batch (same arguments as cch_hull_batched;
 * device buffers, synchronises the stream): coordinate descent over
 * candidate values of each choice, `reps` timed calls per candidate; the
 * fastest goes into the table under this batch's key and into *best (if not
 * NULL).  The outputs hold the batch's hulls afterwards. */
int cch_autotune_batched(const void *points, const int64_t *offsets, int32_t nsets, int32_t dtype,
                         int32_t *out_idx, int32_t *out_counts, void *stream, int32_t reps,
                         cch_tune_params *best);

/* Bytes of device scratch one cch_hull call of this size uses. */
size_t cch_workspace_bytes(int64_t n, int dtype);

/* Free every cached workspace and the servers' pooled pinned host buffers
 * (synchronises the device first). */
void cch_release_workspace(void);

/* ------------------------------------------------------------ serving --
 * A server admits hull requests against a device-memory budget, keeps their
 * inputs and results resident, and batches whatever is admitted into
 * cch_hull_batched launches on a pool of streams, so that requests arriving
 * while others run are started as soon as memory and a stream free up.  Its
 * results are the cch_hull results of each request alone.
 */
typedef struct cch_serve_config {
  size_t budget_bytes;     /* device memory for admitted requests (inputs,
                              outputs and workspaces); 0 -> 64 GiB */
  int32_t num_streams;     /* concurrent batches; 0 -> 4 */
  int32_t max_pending;     /* queue length before CCH_ERR_BUSY; 0 -> 65536 */
  int32_t max_batch;       /* requests per batch; 0 -> 4096 */
  int32_t dtype;           /* CCH_I32 or CCH_F64 for every request */
} cch_serve_config;

typedef struct cch_done {
  uint64_t ticket;
  int32_t status;          /* CCH_OK or a negative code */
  int32_t count;           /* hull size h */
  const int32_t *idx;      /* HOST pointer to the h indices, valid until
                              cch_serve_release(ticket) */
  double latency_ms;       /* submit -> result available */
} cch_done;

typedef struct cch_server cch_server;

/* Create a server (spawns its scheduler thread). */
int cch_serve_create(const cch_serve_config *cfg, cch_server **out);
/* Queue one request; the points (HOST [n,2]) are copied before return.
 * CCH_ERR_RANGE if the request alone exceeds the budget, CCH_ERR_BUSY if
 * the queue is full. */
int cch_serve_submit(cch_server *srv, const void *points, int64_t n, uint64_t *ticket);
/* Queue one request whose points are in DEVICE memory ([n,2] of the
 * server's dtype, 8/16-byte aligned): they are copied, device to device and
 * ordered after the caller's earlier work on `stream`, into a resident
 * buffer the server owns; the copy is complete when the call returns, so the
 * caller may reuse or free its buffer at once.  The request then stays in
 * device memory until its batch has read it (no host copy on the way).  The
 * resident copies of queued requests are not part of the budget, which
 * covers the batches being computed.  Errors as cch_serve_submit. */
int cch_serve_submit_device(cch_server *srv, const void *points, int64_t n, void *stream,
                            uint64_t *ticket);
/* Non-blocking: up to `max` finished requests into done[0 .. *n_done). */
int cch_serve_poll(cch_server *srv, cch_done *done, int max, int *n_done);
/* Free a finished request's result. */
int cch_serve_release(cch_server *srv, uint64_t ticket);
/* Latency and throughput so far: p50/p99 latency (ms) over finished
 * requests, hulls/s since the first submit. */
int cch_serve_stats(cch_server *srv, double *p50_ms, double *p99_ms, double *hulls_per_s,
                    int64_t *finished);
/* Drain in-flight work, stop the scheduler and free everything. */
int cch_serve_destroy(cch_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* CCH_H_ */
