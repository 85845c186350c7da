/*
 * libgwcp — GWCP predictive data-race analysis of a recorded GPU trace, on GB300.
 *
 * The problem (paper "Predictive Data Race Detection for GPUs", sections "Predictive
 * Data Race Detection" and "Extending WCP to GPU Programs"): given one observed trace
 * of a GPU kernel, report the pairs of conflicting accesses that are not ordered by
 * the GWCP partial order. The calls follow that statement: load a trace, compute the
 * order and the race check, report the races.
 *
 * Everything runs on one GPU inside this library (sm_103a kernels); the caller only
 * supplies memory and a CUDA stream. All entry points return 0 on success or a
 * negative GWCP_ERR_* code. No entry point throws or aborts.
 */
#ifndef GWCP_H
#define GWCP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- trace format ---------------------------------------------------------------
 * One 16-byte record per event; trace order is array order. Event kinds follow the
 * paper's event vocabulary (accesses; acquire/release of scoped locks; barriers and
 * warp barriers; fences), section "Tracking GWCP" and Algorithms 1-2.
 *
 *   agent  the analysed thread (a CUDA thread at thread granularity, a warp at warp
 *          granularity); 0 <= agent < num_agents. Block of an agent = agent /
 *          agents_per_block.
 *   op     GWCP_READ, GWCP_WRITE, GWCP_ATOMIC (read-modify-write), GWCP_ACQ, GWCP_REL,
 *          GWCP_BARRIER (one event per barrier instance), GWCP_FENCE.
 *   scope  GWCP_SCOPE_CTA or GWCP_SCOPE_DEVICE for atomics, acquires, releases and
 *          fences; GWCP_SCOPE_CTA or GWCP_SCOPE_WARP for barriers; 0 for READ/WRITE.
 *   space  GWCP_SPACE_GLOBAL or GWCP_SPACE_SHARED (accesses only). Shared locations are
 *          per block (section "Tracking GWCP", shared-memory paragraph).
 *   flags  ignored by the analysis (generators use bit 0 to mark planted events).
 *   addr   accesses: byte address (< 2^63 global, < 2^40 shared); ACQ/REL: lock id;
 *          CTA barrier: the block id it covers; WARP barrier: the lane mask (at thread
 *          granularity the lanes of agent's hardware warp; at warp granularity the
 *          barrier covers the agent alone).
 *
 * Well-formedness (checked on the device; violations give GWCP_ERR_INVALID_TRACE and
 * the first offending index, gwcp_first_bad_index):
 *   W1 fields in range as above;
 *   W2 per agent, a release matches the innermost held acquire (same lock, same scope),
 *      at most 4 locks held at once;
 *   W3 per lock, two critical sections whose scopes overlap (either is device-scoped,
 *      or both are block-scoped in one block) never interleave;
 *   W4 one BARRIER event per barrier instance.
 * Limits of this implementation: n < 2^30 events; num_agents <= 1024, or up to 8192 at
 * GWCP_GRAN_WARP with agents_per_block <= 32 (clocks wider than 1024 entries are kept as
 * tables of 256-entry tiles); a lock may be used with at most 64 scope ids, or 320 when
 * the trace has more than 63 blocks. Other geometries return GWCP_ERR_UNSUPPORTED.
 */
enum {
  GWCP_READ = 0,
  GWCP_WRITE = 1,
  GWCP_ATOMIC = 2,
  GWCP_ACQ = 3,
  GWCP_REL = 4,
  GWCP_BARRIER = 5,
  GWCP_FENCE = 6
};
enum { GWCP_SCOPE_CTA = 0, GWCP_SCOPE_DEVICE = 1, GWCP_SCOPE_WARP = 2 };
enum { GWCP_SPACE_GLOBAL = 0, GWCP_SPACE_SHARED = 1 };
enum { GWCP_GRAN_THREAD = 0, GWCP_GRAN_WARP = 1 };

typedef struct {
  uint32_t agent;
  uint8_t op, scope, space, flags;
  uint64_t addr;
} gwcp_event;

typedef struct {
  uint32_t num_agents;       /* W: width of every vector clock */
  uint32_t agents_per_block; /* num_agents must be a multiple of it */
  uint32_t granularity;      /* GWCP_GRAN_THREAD or GWCP_GRAN_WARP */
  uint32_t reserved;         /* must be 0 */
} gwcp_geometry;

/* A reported race: two event indices, earlier < later. For each access `later` by agent
 * u and each other agent v, `earlier` is the latest access by v before `later` to the
 * same location that conflicts with it (at least one writes; atomics count as writes)
 * and is not exempt (two atomics with overlapping scopes), reported when it is not
 * GWCP-ordered before `later` (section "Tracking GWCP": R_x/W_x checked against C_t).
 * Races are sorted by (later, earlier). */
typedef struct {
  uint64_t earlier, later;
} gwcp_race;

typedef struct {
  uint64_t race_capacity; /* races kept on the device; 0 = max(2^20, n) */
  uint32_t profile;       /* 1 = time each kernel with CUDA events (gwcp_profile_get) */
  uint32_t reserved[5];
} gwcp_options;

typedef struct gwcp_ctx gwcp_ctx; /* opaque; owns all device memory it allocates */

enum {
  GWCP_OK = 0,
  GWCP_ERR_INVALID_TRACE = -1, /* see gwcp_first_bad_index */
  GWCP_ERR_OOM = -2,
  GWCP_ERR_CUDA = -3,
  GWCP_ERR_CAPACITY = -4, /* *n_races still holds the required count */
  GWCP_ERR_TIMEOUT = -5,  /* a bounded device wait gave up; results are void */
  GWCP_ERR_STATE = -6,    /* calls out of order (e.g. report before compute) */
  GWCP_ERR_ARGS = -7,     /* null pointer, bad geometry, size beyond the limits */
  GWCP_ERR_UNSUPPORTED = -8
};

/* Creates a context on CUDA device `device`. opt may be NULL (defaults). */
int gwcp_create(gwcp_ctx** out, int device, const gwcp_options* opt);

/* Makes a trace of n events the context's current trace. ev_is_device = 0: ev is host
 * memory, copied to the device on `cuda_stream` (pinned memory gives an asynchronous
 * copy; the caller must keep ev valid until the stream reaches that point). ev_is_device
 * = 1: ev is device memory read in place by gwcp_compute_order; the caller keeps it
 * valid and unchanged until that work completes. cuda_stream is a cudaStream_t (NULL =
 * legacy default stream). Replaces any previous trace and its results. */
int gwcp_load_trace(gwcp_ctx* ctx, const gwcp_event* ev, uint64_t n, const gwcp_geometry* geo,
                    int ev_is_device, void* cuda_stream);

/* Runs the whole analysis on the device: decode and validation, epoch assignment,
 * critical-section annotation, clock propagation (Algorithms 1-2), access grouping, the
 * per-location race check and race compaction. Kernels are enqueued on cuda_stream; the
 * call synchronises that stream three times: twice to size its buffers from device-side
 * counts and once at the end for the status. Validation errors, a device-side timeout
 * (GWCP_ERR_TIMEOUT) and exhausted device memory (GWCP_ERR_OOM) are returned here and
 * again by gwcp_report_races. */
int gwcp_compute_order(gwcp_ctx* ctx, void* cuda_stream);

/* Waits for the analysis on cuda_stream and copies up to `cap` races into host memory
 * `out` (may be NULL when cap is 0). *n_races receives the total number of races.
 * Returns GWCP_ERR_CAPACITY if cap < total, or if the context's race_capacity was too
 * small (then *n_races is the count required; raise race_capacity and recompute). */
int gwcp_report_races(gwcp_ctx* ctx, gwcp_race* out, uint64_t cap, uint64_t* n_races, void* cuda_stream);

/* Test hook. Copies the clock of event `event_idx` into out_W (num_agents entries):
 * which = 0: C_t of the event's agent (for an access or acquire: after the event's own
 * joins; for a release: the clock it published, before its increment); which = 1: H_t
 * published by a release (GWCP_ERR_UNSUPPORTED for other events). Synchronous. */
int gwcp_debug_clock(gwcp_ctx* ctx, uint64_t event_idx, int which, uint32_t* out_W);

/* Index of the first event that violates W1-W4 after GWCP_ERR_INVALID_TRACE. */
uint64_t gwcp_first_bad_index(const gwcp_ctx* ctx);

/* Profiling (options.profile = 1): after gwcp_report_races, entry i of the last
 * compute's kernel list: its name, device time in ms (CUDA events on the launching
 * stream), and the algorithmic bytes it must move (per the kernel's roofline model).
 * Returns GWCP_ERR_ARGS when i is past the end. */
int gwcp_profile_get(const gwcp_ctx* ctx, int i, const char** name, float* ms, double* bytes);

/* Counters of the last compute: [0] accesses, [1] sync entries (acquire, release and
 * barrier participations), [2] critical sections, [3] in-section accesses, [4] clock
 * versions, [5] partner tests of the check, [6] release-loop record visits,
 * [7] vector-clock joins in the propagation. Synchronous. */
int gwcp_counters(const gwcp_ctx* ctx, uint64_t* out8);

/* Allocation-free analysis of a small trace (the paper has no counterpart: this is an
 * interface for callers that cannot allocate device memory when they need a trace
 * analysed, e.g. code running while another component owns the memory pool, or a hook
 * that must not call cudaMalloc/cudaFree because those can synchronise the device).
 * Same analysis and same results as gwcp_load_trace(ev_is_device = 1) +
 * gwcp_compute_order + gwcp_report_races, but every intermediate buffer comes from one
 * file-scope __device__ scratch array of 96 MiB that every GPU loading the library
 * holds until the process exits; the call itself allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).
 *   ev_dev     device array of n events (read only).
 *   races_dev  device array of races_cap races, written with the first races_cap races
 *              sorted by (later, earlier); may be NULL when races_cap is 0.
 *   n_races    host pointer; receives the total number of races.
 *   first_bad_index  host pointer or NULL; receives the first offending event after
 *              GWCP_ERR_INVALID_TRACE.
 * Limits: n <= 262144 events, num_agents <= 256, and the trace's intermediates must
 * fit the scratch; beyond any of them the call returns GWCP_ERR_UNSUPPORTED and does
 * nothing else. Returns GWCP_ERR_CAPACITY when races_cap < *n_races.
 * Runs on the current CUDA device and synchronises cuda_stream before returning. The
 * first call on a device looks up the scratch array's device address (a one-time
 * set-up per device); make that first call before any stream capture. All calls share
 * the one scratch array: calls that overlap on the GPU (other streams or threads) race
 * on it and must be serialised by the caller. */
int gwcp_analyze_noalloc(const gwcp_event* ev_dev, uint64_t n, const gwcp_geometry* geo, gwcp_race* races_dev,
                         uint64_t races_cap, uint64_t* n_races, uint64_t* first_bad_index, void* cuda_stream);

/* Number of kernels this library has launched in this process, on any context. */
uint64_t gwcp_launch_count(void);

void gwcp_destroy(gwcp_ctx* ctx);
const char* gwcp_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* GWCP_H */
