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
  uint64_t race_capacity; /* races kept on the device; 0 = automatic: max(2^20, n), grown
                             (the check runs again) when a trace has more races */
  uint32_t profile;       /* 1 = time each kernel with CUDA events (gwcp_profile_get) */
  uint32_t blocking_sync; /* 1 = host waits sleep on a blocking-sync event instead of
                             spinning (for many contexts driven by many host threads) */
  uint32_t timeline;      /* 1 = the check records when each of its chunks ends and how many
                             races it found (gwcp_check_timeline) */
  uint32_t hb_only;       /* 1 = the paper's happens-before baseline: accesses are checked
                             against H_t (scoped happens-before of Algorithm 1's H clocks)
                             instead of C_t; C_t <= H_t, so it reports a subset of the
                             GWCP races (the predictable races are the difference) */
  uint32_t pack_walkers;  /* 1 = tile-clock walkers run two CTAs per SM where they fit, which
                             leaves SMs to other streams (fastest alone: 0) */
  uint32_t forced_barrier; /* 1 = forced compression at barriers (section "Vector Clock
                             Compression"): every member of a barrier leaves it at the same
                             local time, the highest N_t among the members, so after the join
                             each member's clock holds one common value for all members.
                             Local times (and the clocks gwcp_debug_clock shows) change; the
                             race set does not. Always on with GWCP_CLOCKS_COMPRESSED */
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
 * counts and once at the end for the status (once more when the automatic race buffer
 * grows and the check runs again; an exhausted tile pool or compressed-version pool is
 * grown and the analysis run again). Buffers are allocated in stream order on
 * cuda_stream from the device's default memory pool and kept for the next call.
 * Validation errors, a device-side timeout (GWCP_ERR_TIMEOUT) and exhausted device
 * memory (GWCP_ERR_OOM) are returned here and again by gwcp_report_races. */
int gwcp_compute_order(gwcp_ctx* ctx, void* cuda_stream);

/* Waits for the analysis on cuda_stream and copies up to `cap` races into host memory
 * `out` (may be NULL when cap is 0): one DMA into page-locked memory, or through the
 * context's own pinned double buffer into pageable memory. *n_races receives the total
 * number of races.
 * Returns GWCP_ERR_CAPACITY if cap < total, or if a fixed race_capacity was too small
 * (then *n_races is the count required; raise race_capacity and recompute). */
int gwcp_report_races(gwcp_ctx* ctx, gwcp_race* out, uint64_t cap, uint64_t* n_races, void* cuda_stream);

/* Test hook. Copies the clock of event `event_idx` into out_W (num_agents entries):
 * which = 0: C_t of the event's agent (for an access or acquire: after the event's own
 * joins; for a release: the clock it published, before its increment); which = 1: H_t
 * published by a release (GWCP_ERR_UNSUPPORTED for other events). Synchronous. */
int gwcp_debug_clock(gwcp_ctx* ctx, uint64_t event_idx, int which, uint32_t* out_W);

/* How clocks are held (the representation only; the race set is identical):
 * GWCP_CLOCKS_DENSE: every clock a row of W words, held in registers by the walker
 *   (num_agents <= 1024; wider traces still use tiles);
 * GWCP_CLOCKS_TILES: clocks as tables of copy-on-write 256-entry tiles (warp granularity,
 *   agents_per_block <= 32, num_agents <= 8192);
 * GWCP_CLOCKS_COMPRESSED: the paper's memory mode (section "Vector Clock Compression"):
 *   the dense walker with forced compression at barriers (options.forced_barrier), and
 *   every clock version the check reads stored in block/warp compressed form - one word
 *   per block when all its entries are equal, else one word per warp (equal entries) or
 *   the warp's 32 values. Release snapshots stay dense. num_agents <= 1024; the check is
 *   the sparse one. gwcp_clock_bytes reports the saving;
 * GWCP_CLOCKS_AUTO (default): tiles from 512 agents on where the trace allows them, else
 *   dense (the two cross near 512 agents on GB300).
 * Applies from the next gwcp_load_trace, which returns GWCP_ERR_UNSUPPORTED when the trace
 * does not allow the requested representation. */
enum { GWCP_CLOCKS_AUTO = 0, GWCP_CLOCKS_DENSE = 1, GWCP_CLOCKS_TILES = 2, GWCP_CLOCKS_COMPRESSED = 3 };
int gwcp_set_clock_mode(gwcp_ctx* ctx, uint32_t mode);

/* How the per-location check visits partners (results are identical):
 * GWCP_CHECK_CHUNKED: one warp per 512-access chunk of the location-sorted accesses keeps
 *   every agent's latest access per class for the current location and tests all of them
 *   for each access (dense clocks only; chunk carries by a segmented max-scan);
 * GWCP_CHECK_SPARSE: accesses grouped by (location, class, agent), in trace order within a
 *   group (one sort of composite keys; with a ranker, a location sort then a regrouping);
 *   locations without a write-class access are left out; each access visits only the
 *   groups of agents that touched its location, each agent once (always used with tile
 *   clocks);
 * GWCP_CHECK_AUTO (default): sparse (measured faster on GB300 at 64-512 warps, 1M-10M
 *   events: 0.54 against 1.90 ms for the check of the 10M-event 64-warp trace).
 * Applies from the next gwcp_compute_order. */
enum { GWCP_CHECK_AUTO = 0, GWCP_CHECK_CHUNKED = 1, GWCP_CHECK_SPARSE = 2 };
int gwcp_set_check_mode(gwcp_ctx* ctx, uint32_t mode);

/* Test hook of failure detection. Every device wait of the analysis (a clock row or
 * barrier count that another walker has not published yet) is bounded: after its poll
 * limit it records GWCP_ERR_TIMEOUT and the walker carries on, so the kernel ends and the
 * context stays usable. This runs that wait in one warp on `device` against a row that
 * nothing ever completes, with `spin_limit` polls; *status receives the kernel's status
 * (GWCP_ERR_TIMEOUT). Synchronous; allocates and frees a small buffer. */
int gwcp_debug_wait_timeout(int device, uint32_t spin_limit, int* status);

/* Test hook of failure detection: caps the bytes of the buffers the context caches
 * (0 = no cap). A compute that would need more fails with GWCP_ERR_OOM, as on an exhausted
 * device, and leaves the context usable: after the cap is raised the next compute runs
 * normally. Host-side only; no device memory is touched. */
int gwcp_debug_alloc_limit(gwcp_ctx* ctx, uint64_t bytes);

/* Index of the first event that violates W1-W4 after GWCP_ERR_INVALID_TRACE. */
uint64_t gwcp_first_bad_index(const gwcp_ctx* ctx);

/* Profiling (options.profile = 1): after gwcp_report_races, entry i of the last
 * compute's kernel list: its name, device time in ms (CUDA events on the launching
 * stream), and the algorithmic bytes it must move (per the kernel's roofline model).
 * Returns GWCP_ERR_ARGS when i is past the end. */
int gwcp_profile_get(const gwcp_ctx* ctx, int i, const char** name, float* ms, double* bytes);

/* Start of profile entry i in ms after the start of entry 0 (the kernels of the side
 * stream overlap those of the main stream: this gives the timeline). GWCP_ERR_ARGS when
 * i is past the end or start_ms is NULL. */
int gwcp_profile_start(const gwcp_ctx* ctx, int i, float* start_ms);

/* Storage of the clock versions of the last compute (the rows the check reads, one per
 * agent and clock-changing step), in bytes: [0] as dense rows of W words (W rounded up to
 * 32 * 2^k), [1] as stored (compressed: headers and written pool words; tiles: tables and
 * tiles handed out; dense: = [0]), [2] as reserved (compressed: headers and the pool
 * chunks the walkers took). Release snapshots are not included. */
int gwcp_clock_bytes(const gwcp_ctx* ctx, uint64_t* out3);

/* Counters of the last compute: [0] accesses, [1] sync entries (acquire, release and
 * barrier participations), [2] critical sections, [3] in-section accesses, [4] clock
 * versions, [5] partner tests of the check, [6] release-loop record visits,
 * [7] vector-clock joins in the propagation. Synchronous. */
int gwcp_counters(const gwcp_ctx* ctx, uint64_t* out8);

/* The counters of gwcp_counters followed by: [8] clock tiles (256 entries, 1 KB) that the
 * propagation's joins and copies read, [9] tiles it wrote (both 0 with dense clocks).
 * Writes the first min(n, GWCP_N_COUNTERS) counters into out (host array). A vector-clock
 * join of width W moves 12 W bytes (two clocks read, one written; the paper's Algorithms
 * 1-2 join full clocks), so [7] x 12 W is the dense join traffic and ([8] + [9]) x 1 KB
 * the traffic of the tiles actually moved. Synchronous. */
#define GWCP_N_COUNTERS 10
int gwcp_counters_ex(const gwcp_ctx* ctx, uint64_t* out, uint32_t n);

/* Allocation-free analysis of a small trace (the paper has no counterpart: this is an
 * interface for callers that cannot allocate device memory when they need a trace
 * analysed, e.g. code running while another component owns the memory pool, or a hook
 * that must not call cudaMalloc/cudaFree because those can synchronise the device).
 * Same analysis and same results as gwcp_load_trace(ev_is_device = 1) +
 * gwcp_compute_order + gwcp_report_races, but every intermediate buffer comes from one
 * file-scope __device__ scratch array of 96 MiB; the call itself allocates nothing (no
 * cudaMalloc, cudaFree or allocating library routine). The array is reserved on a device
 * when the library's device code is loaded there: under CUDA's lazy module loading that
 * is the first call of this function on the device, which a call with n = 0 performs
 * without analysing anything. Make that first call at initialisation (where allocating
 * is allowed) and before any stream capture; the device then holds the array until the
 * process exits.
 *   ev_dev     device array of n events (read only).
 *   races_dev  device array of races_cap races, written with the first races_cap races
 *              sorted by (later, earlier); may be NULL when races_cap is 0.
 *   n_races    host pointer; receives the total number of races.
 *   first_bad_index  host pointer or NULL; receives the first offending event after
 *              GWCP_ERR_INVALID_TRACE.
 * Limits: n <= 262144 events, num_agents <= 256, and the trace's intermediates must
 * fit the scratch; beyond any of them the call returns GWCP_ERR_UNSUPPORTED and does
 * nothing else. Returns GWCP_ERR_CAPACITY when races_cap < *n_races.
 * Runs on the current CUDA device and synchronises cuda_stream before returning, also
 * on an error. Each call looks up the array's device address in the current context.
 * All calls share the one scratch array, which keeps the previous call's contents (each
 * call clears what must start at zero): calls that overlap on the GPU (other streams or
 * threads) race on it and must be serialised by the caller. */
int gwcp_analyze_noalloc(const gwcp_event* ev_dev, uint64_t n, const gwcp_geometry* geo, gwcp_race* races_dev,
                         uint64_t races_cap, uint64_t* n_races, uint64_t* first_bad_index, void* cuda_stream);

/* ---- address ranker --------------------------------------------------------------
 * Not in the paper. A small network scores each location from features of its accesses so
 * that the per-location check visits likely-racy locations first; every location is still
 * checked and the race set does not change. Network: 16 features -> 64 -> 64 -> 1, bfloat16
 * weights and activations with float accumulation; parameters are one float vector of
 * GWCP_RANK_PARAMS values: W1[64][16], b1[64], W2[64][64], b2[64], w3[64], b3.
 * Features of a location (float[16]; its accesses in trace order): log1p of the access,
 * read, write and atomic counts; log1p of the number of distinct agents and blocks (both
 * mod 64); block- and device-scoped atomic fractions; fraction inside a critical section;
 * shared-memory flag; acquire/release/barrier events per trace position over the span
 * from first to last access; log1p(span); share of the first access's agent; agent
 * switches and agent switches with a write or atomic per consecutive pair; fraction of
 * writes and atomics inside a critical section. */
#define GWCP_RANK_PARAMS 5313
#define GWCP_RANK_FEATURES 16

/* Makes the next gwcp_compute_order of ctx check locations in descending score order.
 * theta: host array of GWCP_RANK_PARAMS floats, copied; NULL turns the ranker off. */
int gwcp_set_ranker(gwcp_ctx* ctx, const float* theta);

/* After a successful gwcp_compute_order: the features of every accessed location, in the
 * order the check visited them (ascending location key when no ranker is set), into device
 * arrays feat (cap x GWCP_RANK_FEATURES floats) and keys (cap location keys: the address,
 * or (1 << 63) | (block << 40) | address for shared memory). *n_loc receives the number of
 * locations; GWCP_ERR_CAPACITY when cap < *n_loc. Synchronous on cuda_stream. */
int gwcp_location_features(gwcp_ctx* ctx, float* feat, uint64_t* keys, uint64_t cap, uint64_t* n_loc,
                           void* cuda_stream);

/* Scores of n feature rows (device arrays; theta on the device). Asynchronous. */
int gwcp_rank_scores(const float* theta, const float* feat, uint64_t n, float* scores, void* cuda_stream);

/* Gradient of the mean weighted logistic loss over n rows (labels 0 or 1; positives weighted
 * by pos_weight) with respect to theta, into grad (GWCP_RANK_PARAMS floats) and the loss
 * into *loss (device pointers). The bfloat16 roundings count as the identity. Asynchronous. */
int gwcp_rank_grad(const float* theta, const float* feat, const float* labels, uint64_t n, float pos_weight,
                   float* grad, float* loss, void* cuda_stream);

typedef struct {
  uint32_t epochs, batch; /* passes over the rows; rows per step */
  float lr, pos_weight;   /* Adam step size (beta 0.9 / 0.999, eps 1e-8); weight of label 1 */
  uint32_t reserved[4];
} gwcp_train_options;

/* Trains theta (device, updated in place) with Adam on mini-batches of consecutive rows
 * (shuffle the rows beforehand); epoch_loss (host, may be NULL) receives the mean batch
 * loss of each epoch. One epoch's kernel launches are captured once as a CUDA graph and
 * replayed per epoch (the Adam step count lives on the device). Allocates its optimizer
 * state for the call. Synchronous. */
int gwcp_rank_train(float* theta, const float* feat, const float* labels, uint64_t n, const gwcp_train_options* o,
                    float* epoch_loss, void* cuda_stream);

/* With options.timeline: the check's start (globaltimer ns) and, per chunk of the sorted
 * access stream in check order (512 accesses for the chunked check, 256 for the sparse
 * one), the globaltimer when it ended and the races it found. GWCP_ERR_CAPACITY when
 * cap < *n_chunks. Synchronous. */
int gwcp_check_timeline(gwcp_ctx* ctx, uint64_t* start_ns, uint64_t* chunk_end_ns, uint32_t* chunk_races,
                        uint64_t cap, uint64_t* n_chunks);

/* ---- batched and served analysis: a pool of lanes ----------------------------------
 * The paper analyses one trace at a time. A pool runs many independent traces at once on
 * one GPU: each lane is a context (as gwcp_create) with its own CUDA stream, driven by a
 * host thread of the pool, and runs the same analysis as gwcp_load_trace +
 * gwcp_compute_order + gwcp_report_races; lanes overlap on the device, so short traces
 * and traces whose propagation occupies few SMs share the GPU. Requests are admitted in
 * submission order when a lane is free and the device memory the pool would then hold
 * (every lane's cached buffers plus the new request's estimate) stays within the pool's
 * budget; idle lanes release their buffers when the head request does not fit. A
 * request's race set is identical to the single-context result for the same trace. */
typedef struct {
  const gwcp_event* ev; /* n events, host memory or (ev_is_device = 1) device memory */
  uint64_t n;
  gwcp_geometry geo;
  int32_t ev_is_device;
  uint32_t reserved; /* must be 0 */
} gwcp_trace_desc;

typedef struct {
  uint32_t lanes;         /* worker lanes; 0 = 16. Active lanes start equal to this */
  uint32_t pack_walkers;  /* as gwcp_options.pack_walkers, for every lane */
  uint64_t mem_budget;    /* device bytes the pool may hold; 0 = 85% of free memory at creation */
  uint64_t race_capacity; /* per lane, as gwcp_options.race_capacity */
  uint32_t compress_versions; /* 1 = the paper's memory mode on every lane: traces of up to
                                 1024 agents run with GWCP_CLOCKS_COMPRESSED (forced barrier
                                 compression, compressed clock versions), wider ones with
                                 tiles; the autotuner then leaves the clock modes alone */
  uint32_t reserved[3];   /* must be 0 */
} gwcp_pool_options;

typedef struct {
  int32_t rc;               /* the request's result code (GWCP_OK, or as gwcp_compute_order /
                               gwcp_report_races would return) */
  uint32_t lane;            /* lane that ran it */
  uint64_t n_races;         /* total races (also when the caller's cap was smaller) */
  uint64_t first_bad_index; /* after GWCP_ERR_INVALID_TRACE */
  double t_submit, t_admit, t_done; /* seconds on the pool's steady clock (gwcp_pool_now) */
  double t_first_race;      /* when the check found the request's first race, on the same
                               clock (converted from the GPU's global timer, calibrated
                               to a few microseconds when the pool is created); 0 if the
                               request has no race or failed. t_done comes later by the rest
                               of the check, the race sort and the copy of the races */
} gwcp_request_info;

typedef struct gwcp_pool gwcp_pool; /* opaque; owns its lanes, threads and device memory */

/* Creates a pool on `device`; opt may be NULL (defaults). */
int gwcp_pool_create(gwcp_pool** out, int device, const gwcp_pool_options* opt);

/* Queues one trace. The pool keeps the pointers: `t->ev` must stay valid and unchanged,
 * and `out` (host memory, `cap` races, may be NULL when cap is 0) writable, until the
 * request has been waited for. *ticket identifies the request. Never blocks on the GPU. */
int gwcp_pool_submit(gwcp_pool* p, const gwcp_trace_desc* t, gwcp_race* out, uint64_t cap, uint64_t* ticket);

/* Result of a request. block = 1 waits for it; block = 0 returns 1 if it is still queued
 * or running. On completion returns 0 and fills *info (may be NULL); the ticket is then
 * released. GWCP_ERR_ARGS for an unknown ticket. The request's own code is info->rc. */
int gwcp_pool_wait(gwcp_pool* p, uint64_t ticket, int block, gwcp_request_info* info);

/* Analyses n traces and waits for all: submits them longest first (so long traces do
 * not end up alone at the tail), then fills n_races[i] and rc[i] (either may be NULL)
 * and writes up to cap[i] races into out[i] (out may be NULL when every cap is 0).
 * Returns 0, or the first nonzero rc[i]. */
int gwcp_pool_run_batch(gwcp_pool* p, const gwcp_trace_desc* t, uint32_t n, gwcp_race* const* out,
                        const uint64_t* cap, uint64_t* n_races, int32_t* rc);

/* Number of lanes that take requests (1..lanes given at creation). */
int gwcp_pool_set_active_lanes(gwcp_pool* p, uint32_t active);

/* Autotuner. First, for every clock-width class (ceil(log2(num_agents))) among the n
 * traces whose traces all allow both clock representations (gwcp_set_clock_mode), times
 * them one after another with dense and with tile clocks and keeps the faster for that
 * class (gwcp_pool_clock_modes). Then runs the n traces as one batch with each candidate
 * number of active lanes (1, 2, 4, 8, 12, 16, 24, 32, up to the pool's lanes), keeps the
 * largest whose time is within 5% of the fastest (near the optimum the times differ by
 * about that much from run to run, and more lanes overlap more requests that arrive over
 * time) and returns it in *best (seconds per candidate in secs[], up to 8 entries, may
 * be NULL). Last, with that many lanes, runs the batch once more with the other setting
 * of pack_walkers and keeps whichever was faster (gwcp_pool_settings). Races are counted,
 * not copied. */
int gwcp_pool_autotune(gwcp_pool* p, const gwcp_trace_desc* t, uint32_t n, uint32_t* best, double* secs);

/* The pool's current settings: active lanes and whether tile walkers are packed two CTAs
 * per SM (the autotuner's choices, or the creation options). Either pointer may be NULL. */
int gwcp_pool_settings(const gwcp_pool* p, uint32_t* active_lanes, uint32_t* pack_walkers);

/* The clock mode the pool uses per width class c = ceil(log2(num_agents)), c < 16
 * (GWCP_CLOCKS_AUTO where the autotuner has not chosen). */
int gwcp_pool_clock_modes(const gwcp_pool* p, uint32_t* modes16);

/* Seconds on the pool's steady clock (the clock of gwcp_request_info). */
double gwcp_pool_now(const gwcp_pool* p);

/* Device bytes the pool's lanes hold now. */
uint64_t gwcp_pool_device_bytes(gwcp_pool* p);

/* Waits for every queued request, stops the threads, frees everything. Requests not yet
 * waited for are dropped. */
void gwcp_pool_destroy(gwcp_pool* p);

/* Number of kernels this library has launched in this process, on any context (a kernel
 * in a replayed CUDA graph counts once, when it was captured). */
uint64_t gwcp_launch_count(void);

void gwcp_destroy(gwcp_ctx* ctx);
const char* gwcp_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* GWCP_H */
