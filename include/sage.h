/*
 * sage.h -- C-ABI of a B300-native runtime for many concurrent invocations of
 * one GPU function that share one reference-counted device copy of the
 * function's read-only data (SAGE, arXiv 2404.14691).
 *
 * Paper mapping
 *   - Request / Data{key, Type ReadOnly|Writable, data_dptr} (Sec. 4.2, Sec. 5.1,
 *     Sec. 6.2): sage_fn_desc / sage_data_desc / sage_access.
 *   - Unified memory daemon, one per GPU, that loads data proactively and hands
 *     out device addresses (Sec. 4.1, Sec. 5.1): sage_pool.
 *   - Parallelised function setup: GPU data preparation runs beside the context /
 *     module / workspace setup (Sec. 5.1, stages 3||4 and 5||6 of fig. workflow):
 *     sage_prepare returns at once; staging runs on the pool's side stream and
 *     host producer threads while the calling thread loads kernels and builds the
 *     workspace.
 *   - SageLoadToGPU returns the pointer before the data is ready; the kernel
 *     executor checks readiness before launch (Sec. 5.2): sage_invoke makes the
 *     launch stream wait on the data's ready event; sage_wait is the host-side
 *     form of the same check.
 *   - Read-only memory sharing (Sec. 6.2): a second sage_prepare of the same key
 *     takes a reference to the resident copy and loads nothing.
 *   - Multi-stage resource exit (Sec. 6.3): sage_release frees (or, with a host
 *     cache, demotes to host memory) a key's read-only data after its last
 *     reference; sage_pool_destroy ends the daemon.
 *   - Memory taxonomy (Sec. 6.1, Table tb:memory): sage_pool_stats separates the
 *     read-only bytes from the workspaces (writable memory).
 *   - Context memory sharing (Sec. 6.4): every invocation of a function runs in
 *     one process / one CUDA context and reuses its kernels and workspace.
 *
 * The GPU function (the workload this runtime executes; the paper names no
 * specific one) is a recommendation-style inference per sample b:
 *     pooled[b, t*D:(t+1)*D] = sum over bag (t,b) of table_t rows
 *     h = ReLU(... ReLU(x_b W0^T + b0) ...)              bottom MLP
 *     c = [pooled[b, 0:T*D], h]                           concat
 *     out[b] = sigmoid(top MLP(c)), ReLU after hidden top layers, last layer linear
 *
 * Conventions
 *   - All functions return a sage_status; none throws or aborts.  On an error
 *     sage_last_error() returns a thread-local message.
 *   - "device" pointers are addresses in the pool's CUDA device; "host" pointers
 *     are CPU addresses (pinned memory is faster but not required).
 *   - Streams are cudaStream_t passed as void*; NULL means the legacy default stream.
 *   - The library is thread-safe: a pool is protected by a mutex; invocations of
 *     the same or different functions may be issued from any threads on any streams.
 */
#ifndef SAGE_H
#define SAGE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sage_pool_s* sage_pool;
typedef struct sage_fn_s* sage_fn;

typedef enum {
    SAGE_OK = 0,
    SAGE_PENDING = 1,          /* sage_fn_query: staging not finished yet (not an error) */
    SAGE_ERR_INVALID = -1,     /* bad argument, or a key re-prepared with another shape */
    SAGE_ERR_NOMEM = -2,       /* the pool's device-memory budget (or the device) is exhausted */
    SAGE_ERR_CUDA = -3,        /* a CUDA call failed; see sage_last_error() */
    SAGE_ERR_TIMEOUT = -4,     /* a bounded host wait ran out */
    SAGE_ERR_BUSY = -5,        /* sage_pool_destroy with live references */
    SAGE_ERR_STAGING = -6,     /* the producer of the read-only data failed; the handle is sticky-failed */
    SAGE_ERR_BOUNDS = -7,      /* a kernel saw a bag row index outside its table (reported by sage_fn_check) */
    SAGE_ERR_DEVICE = -8       /* a kernel's bounded wait ran out (reported by sage_fn_check) */
} sage_status;

/* Data.Type of the paper (Sec. 6.2): read-only data is shared between invocations. */
typedef enum { SAGE_READONLY = 0, SAGE_WRITABLE = 1 } sage_access;

/* Element type of the function's tables and weights.  SAGE_F32: fp32 tables,
 * weights and activations.  SAGE_BF16: bf16 tables, weights and activations,
 * fp32 accumulation on the tensor cores, fp32 biases, fp32 dense input. */
typedef enum { SAGE_F32 = 0, SAGE_BF16 = 1 } sage_dtype;

/* Device allocator hooks.  dev_alloc returns device memory of `bytes` usable on
 * `stream` (a cudaStream_t) or NULL; dev_free returns it.  When both are NULL the
 * pool uses cudaMallocAsync / cudaFreeAsync on its own side stream.  A Python
 * caller may pass PyTorch's caching allocator here. */
typedef void* (*sage_dev_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*sage_dev_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);

typedef struct {
    int device;                    /* CUDA ordinal; pools on several devices may share a process */
    size_t budget_bytes;           /* device bytes the pool may hold for read-only data and
                                      workspaces; 0 = free memory at creation minus 2 GiB */
    size_t staging_chunk_bytes;    /* pinned staging chunk size; 0 = 64 MiB (rounded to 4 KiB) */
    int staging_chunks;            /* pinned chunks in the ring; 0 = 4 */
    int producer_threads;          /* host threads filling each chunk; 0 = min(16, cores) */
    int serial_setup;              /* 1 = sage_prepare waits for staging before module /
                                      workspace setup (the non-overlapped form, for comparison) */
    sage_dev_alloc_fn dev_alloc;   /* optional */
    sage_dev_free_fn dev_free;     /* optional; set both or neither */
    void* alloc_ctx;
    size_t host_cache_bytes;       /* stage 2 of the multi-stage exit (Sec. 6.3): when the last
                                      reference of a key is released, its read-only data is kept in
                                      page-locked host memory (up to this many bytes, least recently
                                      used images evicted) and a later prepare of the key re-stages
                                      from there at link speed instead of calling its producer.
                                      0 = off (release frees everything). */
    int graphs;                    /* 1 = sage_invoke / sage_invoke_batch capture each batch's launch
                                      chain into a CUDA graph (updated in place while the kernels stay
                                      the same) and launch it in one call; 0 = direct launches.  Host-buffer
                                      batches (and sage_serve) and streams of an SM partition always launch
                                      directly */
    int exportable;                /* 1 = read-only items are allocated as exportable physical memory
                                      (CUDA virtual memory management, POSIX file-descriptor handles)
                                      so that sage_share_start can map them into other processes;
                                      dev_alloc is then used for workspaces only */
} sage_pool_config;

/* Producer of a data item: fill bytes [offset, offset+bytes) of the item into the
 * host buffer dst.  offset and bytes are multiples of 256 except at the item's end.
 * May be called concurrently from several host threads on disjoint ranges.
 * Returns 0 on success, nonzero on failure (the item becomes sticky-failed). */
typedef int (*sage_fill_fn)(void* dst, size_t offset, size_t bytes, void* ctx);

/* One data item of a request (Data of Sec. 5.1 / 6.2).  Exactly one of host_src
 * or fill must be set.  The caller keeps host_src (or fill_ctx) alive until
 * sage_wait returns SAGE_OK for a handle of this key (or the handle fails). */
typedef struct {
    const char* key;               /* unused for the two items of sage_fn_desc (the fn_key names both) */
    sage_access access;            /* must be SAGE_READONLY for tables and weights */
    size_t bytes;
    const void* host_src;          /* host image of the item, or NULL */
    sage_fill_fn fill;             /* producer, or NULL */
    void* fill_ctx;
} sage_data_desc;

/* A GPU function: its shape and its read-only data.
 *
 * tables item: the T tables back to back, table t = rows[t] x dim elements of
 *   `dtype`, row-major, no padding (bytes = sum(rows) * dim * elem).
 * weights item: for each layer l in order (bottom layers, then top layers):
 *   W_l [out_l x in_l] of `dtype`, row-major, then b_l [out_l] fp32; each of the
 *   two arrays starts at a 256-byte aligned offset from the start of the item;
 *   bytes = the end of the last bias rounded up to 256.
 *   Bottom layer 0 has in = n_dense; top layer 0 has in = num_tables*dim +
 *   bot_dims[n_bot-1]; the last top layer has out = 1.
 * Limits: 1 <= num_tables <= 128; dim*elem a power of two in [16, 1024] bytes;
 *   1 <= n_dense <= 64; n_bot, n_top in [1, 8]; for SAGE_BF16 every layer but
 *   bottom 0 and the last top layer needs in and out multiples of 64 (tensor-core
 *   tiles); rows[t] < 2^31. */
typedef struct {
    const char* fn_key;            /* identity of the read-only data (Data.key) */
    sage_dtype dtype;
    int num_tables;
    const int64_t* rows;           /* [num_tables] */
    int dim;
    int n_dense;
    int n_bot;
    const int* bot_dims;           /* [n_bot] output sizes */
    int n_top;
    const int* top_dims;           /* [n_top] output sizes, last == 1 */
    int max_batch;                 /* samples per workspace slot at prepare (grown on demand); 0 = 4096 */
    int workspace_slots;           /* invocations in flight per function; 0 = 2 */
    sage_data_desc tables;
    sage_data_desc weights;
} sage_fn_desc;

/* One invocation (a request's writable data, all in device memory). */
typedef struct {
    int batch;                     /* B >= 0 samples */
    const float* dense;            /* device [B, n_dense] fp32 row-major */
    const int32_t* indices;        /* device: row indices of all bags */
    const int64_t* offsets;        /* device [num_tables*B + 1], table-major CSR: bag (t,b) is
                                      indices[offsets[t*B+b] .. offsets[t*B+b+1]) */
    float* out;                    /* device [B]: sigmoid outputs */
    int64_t num_indices;           /* optional: offsets[T*B] - offsets[0] when known on the host, else 0;
                                      used only for the byte count of the kernel-timing record */
} sage_invocation;
/* The device offsets are read only by the kernels, never on the host, so they are
 * not checked: they must never decrease and must stay inside the indices buffer
 * (a bad offset reads outside the caller's indices).  Row indices outside their
 * table are checked on the device (skipped, SAGE_ERR_BOUNDS from sage_fn_check). */

/* The same invocation with HOST buffers (Writable data loaded to the GPU and the
 * result dumped back, SageLoadToGPU / SageDumpToDB of Sec. 5.2). */
typedef struct {
    int batch;
    const float* dense;            /* host [B, n_dense] */
    const int32_t* indices;        /* host [num_indices] */
    const int64_t* offsets;        /* host [num_tables*B + 1], offsets[0] == 0 */
    int64_t num_indices;           /* == offsets[num_tables*B] */
    float* out;                    /* host [B] */
} sage_host_invocation;
/* Host offsets are checked before anything is copied: offsets[0] == 0, never
 * decreasing, offsets[num_tables*B] == num_indices; otherwise the call (and
 * sage_serve, for any request) returns SAGE_ERR_INVALID. */

typedef struct {
    size_t budget_bytes;
    size_t resident_bytes;         /* read-only data + workspaces currently held */
    size_t readonly_bytes;         /* read-only data currently held */
    int64_t functions;             /* resident function entries */
    int64_t refs;                  /* live handles over all entries */
    int64_t h2d_bytes;             /* read-only bytes staged host->device since creation */
    int64_t prepares, hits, misses;
    int64_t invocations;           /* invocations issued (a batch counts its members) */
    int64_t launches;              /* kernels launched by the library */
    double ctx_ms;                 /* context + pool creation time */
    double last_stage_ms;          /* host time from prepare to the last chunk enqueued (last miss) */
    double last_fill_ms;           /* producer time inside that staging */
    double last_module_ms;         /* kernel loading + attribute setup of the last miss */
    double last_workspace_ms;      /* workspace allocation + tensor-map setup of the last miss */
    double last_prepare_ms;        /* wall time of the last sage_prepare call */
    size_t host_cache_bytes;       /* read-only images held in the host cache */
    int64_t host_cache_entries;
    int64_t host_cache_hits;       /* prepares re-staged from the host cache */
    int64_t demotions;             /* releases that moved read-only data to the host cache */
} sage_pool_stats_t;

/* Create a pool on config->device: makes the CUDA context current, creates the
 * side (staging) stream, the pinned staging ring and the producer threads.
 * Paper: the unified memory daemon, one per GPU (Sec. 4.1), set up by SageInit
 * (Sec. 4.2).  config may be NULL (defaults).  On failure *out is untouched;
 * SAGE_ERR_CUDA when the device or its context cannot be set up. */
sage_status sage_pool_create(const sage_pool_config* config, sage_pool* out);

/* Prepare function desc->fn_key and return a new reference in *out.
 * Resident key: takes a reference (no data loaded) -- read-only sharing, Sec. 6.2.
 * New key: reserves budget (SAGE_ERR_NOMEM if over), allocates the device copy,
 * queues the staging of tables and weights, then -- on the calling thread, while
 * staging runs -- loads the kernels and allocates the workspace (the engine's
 * context preparation beside the daemon's data preparation, Sec. 5.1).
 * Returns without waiting for the data.  A resident key re-prepared with another
 * dtype, shape or byte size returns SAGE_ERR_INVALID. */
sage_status sage_prepare(sage_pool pool, const sage_fn_desc* desc, sage_fn* out);

/* Device addresses of the function's read-only items (data_dptr of Sec. 5.1 /
 * SageLoadToGPU of Sec. 5.2): valid while the handle lives; the bytes are there
 * only once sage_fn_query / sage_wait return SAGE_OK (kernels launched by
 * sage_invoke* wait for them on the device).  Either output may be NULL. */
sage_status sage_fn_data(sage_fn fn, const void** tables, const void** weights);

/* Non-blocking readiness query: SAGE_OK when the read-only data is on the device,
 * SAGE_PENDING while staging, SAGE_ERR_STAGING after a producer failure. */
sage_status sage_fn_query(sage_fn fn);

/* Wait on the host until the function's read-only data is on the device.
 * Paper: SageLoadToGPU hands out the pointer before the data has arrived, and
 * the kernel executor asks the daemon whether the data is ready before it
 * launches (Sec. 5.2); sage_fn_data is the first half, this call the host-side
 * form of the second (sage_invoke* need not call it: they make the device wait).
 * timeout_us < 0 waits forever.  Returns SAGE_OK, SAGE_ERR_TIMEOUT (the data is
 * still being staged; the handle stays usable) or SAGE_ERR_STAGING (the producer
 * failed; sticky); SAGE_ERR_INVALID for a bad handle. */
sage_status sage_wait(sage_fn fn, int64_t timeout_us);

/* Run one invocation on `stream` (asynchronous): SageRun of Sec. 4.2 for one
 * request.  The stream first waits, on the device, for the read-only data (the
 * executor's readiness check, Sec. 5.2); the
 * calling thread blocks only until the last staging copy has been queued.
 * Returns SAGE_ERR_STAGING if the data failed to load. */
sage_status sage_invoke(sage_fn fn, const sage_invocation* inv, void* stream);

/* Run n invocations of the same function as ONE fused batch of sum(batch) samples
 * on `stream`: one launch per layer / gather over all of them, outputs written to
 * each invocation's own `out`.  Each result equals (bitwise) the result of
 * invoking it alone.  The paper has no counterpart (batching is this library's
 * addition); n in [1, 256], the buffers of every invocation as for sage_invoke. */
sage_status sage_invoke_batch(sage_fn fn, const sage_invocation* invs, int n, void* stream);

/* sage_invoke_batch with host buffers: copies each invocation's inputs to the
 * device, runs the fused batch and copies the outputs back, all on `stream`;
 * returns after the outputs are in host memory. */
sage_status sage_invoke_batch_host(sage_fn fn, const sage_host_invocation* invs, int n, void* stream);

/* sage_invoke_batch_host without the final wait: enqueues the input copies, the
 * fused batch and the output copies and returns.  The inputs are copied on the
 * workspace slot's own copy stream, which waits only for that slot's previous
 * batch, so with workspace_slots >= 2 consecutive calls overlap one batch's
 * copies with the previous batch's compute.  The host buffers must stay valid,
 * and the outputs may be read, only after `stream` has been synchronised. */
sage_status sage_invoke_batch_host_async(sage_fn fn, const sage_host_invocation* invs, int n, void* stream);

/* Read and clear the function's device error word after synchronising it:
 * SAGE_OK, SAGE_ERR_BOUNDS (a bag row index was outside its table; the row was
 * skipped) or SAGE_ERR_DEVICE (a kernel's bounded wait ran out). */
sage_status sage_fn_check(sage_fn fn);

/* Test read-back: copy one activation buffer of the most recent batch that ran on
 * this function's key (any handle, any sage_invoke* call) to host memory `dst`,
 * after waiting for that batch.  which = 0: the concat buffer [M, T*dim +
 * bot_dims[n_bot-1]] (the gather's pooled columns, then the bottom MLP's output);
 * which = 1 + l: the output of top hidden layer l [M, top_dims[l]], l < n_top - 1,
 * when it is written (SAGE_ERR_INVALID for the last hidden layer when the sigmoid
 * head runs in its epilogue).  Rows are the batch's samples in invocation order.
 * plane 0: the values as stored (fp32; bf16 for SAGE_BF16 functions; for fp32
 * functions whose hidden layers run on the tensor cores, the tf32-rounded "hi"
 * part), plane 1: the fp32 residual "lo" of such functions (value = hi + lo
 * exactly), else SAGE_ERR_INVALID.  bytes must be M * width * element size.
 * *rows_out (may be NULL) receives M; with dst NULL nothing is copied.  A later
 * batch may reuse the workspace: call it before the next batch.  The paper has no
 * counterpart (it lets tests compare intermediate results with the oracle). */
sage_status sage_fn_debug_copy(sage_fn fn, int which, int plane, void* dst, size_t bytes, int* rows_out);

/* Drop a reference (the handle is invalid afterwards).  When the last reference
 * of a key is dropped, the pool waits for the key's in-flight work, frees its
 * device copy and workspace and returns the budget -- or, with host_cache_bytes,
 * first keeps the read-only data in host memory: the first two stages of the
 * paper's multi-stage resource exit (Sec. 6.3).  SAGE_ERR_INVALID for a bad
 * handle; SAGE_ERR_CUDA when waiting for that work reported a device failure that
 * no earlier call had surfaced (the memory and the handle are released anyway). */
sage_status sage_release(sage_fn fn);

/* Destroy an empty pool: the daemon's end, after every function it served has
 * exited (the last stage of Sec. 6.3).  SAGE_ERR_BUSY while any reference is
 * live (nothing is freed then); the host cache is freed.  SAGE_ERR_CUDA when the
 * pool's last staging or allocation work reported a device failure (the pool is
 * destroyed anyway). */
sage_status sage_pool_destroy(sage_pool pool);

/* Copy the pool's counters into *out.  Read-only bytes and workspace bytes are
 * counted apart, the paper's split of a function's memory into read-only,
 * writable and context memory (Sec. 6.1, Table tb:memory); H2D bytes count each
 * shared key once (Sec. 6.2).  SAGE_ERR_INVALID for a NULL argument. */
sage_status sage_pool_stats(sage_pool pool, sage_pool_stats_t* out);

/* Page-locked host memory for invocation buffers and host images: 2 MiB aligned,
 * backed by transparent huge pages where the kernel allows, registered with
 * cudaHostRegister (rounded up to 2 MiB).  Host->device copies from it run near
 * the link rate even for buffers of a few MB, which small separately pinned
 * allocations do not on hosts that map DMA through 4 KiB pages.  Free with
 * sage_host_free. */
sage_status sage_host_alloc(size_t bytes, void** out);
sage_status sage_host_free(void* ptr);

/* Thread-local message of the last error returned on this thread ("" if none).
 * The paper has no counterpart (status codes replace exceptions at the boundary). */
const char* sage_last_error(void);

/* Number of kernels the library has launched in this process (all pools). */
int64_t sage_kernel_launches(void);

/* Kernel timing.  While enabled, every kernel that sage_invoke* launches is
 * bracketed by two timing CUDA events recorded on the stream it is launched on.
 * sage_profile_read synchronises those events, aggregates them per kernel kind
 * (names: "bottom0", "gemm_f32", "gemm_tc", "gemm_tf32x3", "gather", "head") into out[0..max)
 * and clears the record; it returns the number of kinds written (or a negative
 * sage_status).  Enabling adds two event records per kernel to the stream and
 * runs the bottom MLP on the launch stream instead of beside the gather, so that
 * every kernel's events time it alone. */
typedef struct {
    char name[16];
    int64_t launches;
    double total_ms;
    double work;                   /* algorithmic bytes (gather) or flops (GEMMs) summed over launches */
} sage_kernel_time;

sage_status sage_profile_enable(int on);
int sage_profile_read(sage_kernel_time* out, int max);

/* ---- autotuning of the tensor-core GEMM tiles ----
 * sage_autotune times every tile configuration (N tile x pipeline depth) of each
 * tensor-core layer of `fn` for a batch of `rows` samples (bucketed to the next
 * power of two) on scratch operands it allocates and frees, and records the
 * fastest per shape in a process-wide table that every later launch of that
 * shape uses; for an fp32 function whose bottom layers 0 and 1 can run as one
 * kernel it also times that kernel against the two separate ones.  Synchronous.  sage_tuning_save / _load write / read the table as
 * text keyed by the GPU's name (entries for other GPUs are ignored on load). */
sage_status sage_autotune(sage_fn fn, int rows, void* stream);
/* Pin a tile configuration for GEMM shape (kind, batch rows bucket, N, K): kind 1 =
 * BF16, 2 = fp32 splitting in shared memory, 3 = fp32 from pre-split planes (the
 * fp32 functions' path; stages >= 100 selects the persistent kernel with stages-100
 * pipeline stages), 4 = bottom layers 0 and 1 of an fp32 function in one kernel
 * (N = layer 1's outputs, K = layer 0's outputs; (bn, stages) = (256, 102),
 * (128, 103) or (64, 104), or (1, 1) for separate kernels; fusable when layer 0
 * has at most 15 inputs and at most 512 outputs, a multiple of 32, and every
 * hidden layer runs on the tensor cores; untuned, fusable shapes run fused).
 * SAGE_ERR_INVALID for configurations the kernel does not have. */
sage_status sage_tuning_set(int kind, int rows, int N, int K, int bn, int stages);
sage_status sage_tuning_save(const char* path);
sage_status sage_tuning_load(const char* path);

/* ---- serving ----
 * sage_serve replays a trace of timed requests against several functions on the
 * pool's GPU with continuous batching (the project's serving form; the paper's
 * evaluation replays a trace of function requests, Sec. 7.1).  Each function is
 * prepared when its first request arrives (cold setup: staging beside kernel
 * loading, Sec. 5.1) and its requests queue until its data is ready.  Admission
 * is by device memory: a prepare that exceeds the pool budget evicts idle
 * resident functions (least recently used first) or waits.  Every function owns
 * lanes_per_fn streams, each with its own workspace slot; the queued requests of
 * a function are split evenly over its idle lanes and each lane runs its share
 * (up to the batch limits) as one fused batch, so requests arriving while others
 * run join the next batches, and lanes overlap on the device.  An idle function keeps its data
 * for linger_s (stage 1 of the multi-stage exit, Sec. 6.3), then is released.
 * Request buffers are host memory (pinned recommended): inputs are copied in and
 * outputs copied back inside each batch.  Latency = completion - arrival. */
typedef struct {
    int fn;                        /* index into fns[] */
    double arrival_s;              /* arrival time, seconds from the start of the replay */
    sage_host_invocation inv;      /* the request's host buffers */
} sage_request;

typedef struct {
    int max_batch_invocations;     /* requests per fused batch, <= 256; 0 = 256 */
    int64_t max_batch_rows;        /* samples per fused batch; 0 = 65536 (a single larger request still runs) */
    int lanes_per_fn;              /* concurrent batches per function; 0 = 2 */
    double linger_s;               /* keep an idle function resident this long; < 0 = until evicted */
    double timeout_s;              /* give up after this long (SAGE_ERR_TIMEOUT); 0 = 600 */
    int sm_partition;              /* 1 = each function's lanes run in its own SM partition (one green
                                      context per function, SMs / n_fns each, see sage_partition_create);
                                      0 = all functions share every SM */
} sage_serve_config;

typedef struct {
    double latency_ms;             /* completion - arrival (-1 if it did not complete) */
    double queue_ms;               /* launch - arrival: queueing incl. waiting for a cold setup */
    double service_ms;             /* completion - launch */
    int cold;                      /* 1: its function was not resident and ready when it arrived */
    int batch_invocations;         /* requests fused into its batch */
    int status;                    /* sage_status of this request */
} sage_request_result;

typedef struct {
    double wall_s;
    int64_t completed, batches, prepares, evictions, cold_requests, max_inflight_batches;
    double invocations_per_s;      /* completed / wall_s */
    double mean_ms, p50_ms, p99_ms, warm_p50_ms, warm_p99_ms, cold_p50_ms, cold_p99_ms;
} sage_serve_stats;

/* fns[]: the functions (their data items must stay valid for the whole replay);
 * reqs[]: n requests (any order); results[]: n outputs (required); stats may be
 * NULL.  Returns SAGE_OK when every request completed, else the first error. */
sage_status sage_serve(sage_pool pool, const sage_fn_desc* fns, int n_fns, const sage_request* reqs, int n,
                       const sage_serve_config* config, sage_request_result* results, sage_serve_stats* stats);

/* ---- invocation without any device allocation ----
 * The paper has no counterpart of this entry point.  It serves callers that may
 * not allocate device memory at all -- a latency-critical host thread that must
 * never enter the device allocator, or a runtime that owns every device byte
 * itself -- and so cannot hold a sage_fn, whose workspace the pool allocates.
 * It runs one invocation exactly like sage_invoke (same kernels, same results
 * within the same tolerances), but takes the function's shape (`shape`; its two
 * data items are ignored) and its read-only data as caller-owned device
 * pointers: `tables` and `weights` laid out as the tables / weights items of
 * sage_fn_desc.  The caller passes inputs and outputs in `inv` as for sage_invoke.
 * Its activations and error word live in one static device array of 64 MiB that
 * every GPU loading this library holds until exit; a batch whose activations do
 * not fit is rejected with SAGE_ERR_INVALID and a message giving the bytes
 * needed.  It calls no allocator (no cudaMalloc/cudaMallocAsync/cudaFree, no
 * library routine that allocates).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current; make
 * that first call before any stream capture.  The address is cached for the
 * life of the process: resetting the device after the first call is not
 * supported.  All calls share the array and it keeps the last call's contents:
 * calls whose kernels overlap on the GPU race, so issue them on one stream (or
 * order them).  Alignment: tables and weights 256 bytes, dense and out 16 bytes,
 * indices 4 bytes, offsets 8 bytes; a misaligned pointer is refused with
 * SAGE_ERR_INVALID before anything is launched.  Out-of-range bag rows are
 * skipped, and a tensor-core GEMM whose bounded wait runs out leaves its output
 * wrong; both set the array's error word, which each call clears first and
 * sage_noalloc_check reports.  Asynchronous on `stream`. */
sage_status sage_invoke_noalloc(const sage_fn_desc* shape, const void* tables, const void* weights,
                                const sage_invocation* inv, void* stream);

/* Error report of the no-allocation entry point on the current device: waits for
 * `stream` (the stream of the calls to check), reads the shared error word into
 * host memory and clears it (no allocation).  Returns SAGE_OK, SAGE_ERR_BOUNDS (a
 * bag row index was outside its table; that row was skipped) or SAGE_ERR_DEVICE
 * (a kernel's bounded wait ran out; the outputs of that call are not valid).
 * Every call clears the word when it starts, so the report covers the last call
 * on `stream`: check after each call whose errors matter.  The paper has no
 * counterpart. */
sage_status sage_noalloc_check(void* stream);

/* ---- building blocks (the kernels of sage_invoke, callable one by one) ----
 * Used by the parity tests and the kernel benchmarks.  All pointers are device
 * pointers; all calls are asynchronous on `stream`; err_word (device int, may be
 * NULL) receives bit 1 on an out-of-range row and bit 2 on a timed-out wait. */

/* Embedding-bag sum (the gather of the function):
 *   out[b*ldo + t*dim + d] = sum_{i in [offsets[t*B+b], offsets[t*B+b+1])} table_t[indices[i]*dim + d]
 * tables: the tables item (back to back, `dtype`); table_rows [T] on the host;
 * out: fp32 for SAGE_F32, bf16 (round to nearest even) for SAGE_BF16, row stride
 * ldo elements.  Sums run in fp32 in a fixed order (independent of B).
 * uniform-length bags, index layout and ranges as in sage_invocation. */
sage_status sage_embedding_bag_sum(sage_dtype dtype, const void* tables, const int64_t* table_rows,
                                   int num_tables, int dim, int batch, const int32_t* indices,
                                   const int64_t* offsets, void* out, int ldo, int* err_word,
                                   void* stream);

/* Linear layer y = act(x W^T + bias) for M rows: x [M, K] (row stride ldx),
 * W [N, K] row-major, bias [N] fp32, y [M, N] (row stride ldy); act 0 = none,
 * 1 = ReLU.  SAGE_F32: fp32 in/out; when N is a multiple of 64 (and rows are
 * 16-byte aligned) on the tensor cores as three tf32 products of the hi/lo split
 * of x and W (error below ~3*2^-22 * sum|x||w|), else fp32 FMA.  SAGE_BF16:
 * bf16 in/out, tcgen05 tensor cores with fp32 accumulation in tensor memory;
 * needs K and N multiples of 64 and 16-byte aligned rows. */
sage_status sage_linear(sage_dtype dtype, int M, int N, int K, const void* x, int ldx, const void* W,
                        const float* bias, int act, void* y, int ldy, int* err_word, void* stream);

/* sage_linear with an explicit tensor-core tile configuration: N tile `bn` and
 * pipeline depth `stages` (0, 0 = automatic / tuned).  Configurations: BF16
 * (256,4) (128,6) (64,8) (256,2) (128,3) (64,4); F32 on tensor cores (128,3)
 * (64,4) (64,2).  SAGE_ERR_INVALID for other pairs or shapes they cannot tile. */
sage_status sage_linear_tiled(sage_dtype dtype, int M, int N, int K, const void* x, int ldx, const void* W,
                              const float* bias, int act, void* y, int ldy, int bn, int stages, int* err_word,
                              void* stream);

/* ---------------------------------------------------------------- cross-process sharing
 *
 * The paper's memory daemon is a separate process: a function's engine hands it
 * the data request first, and the daemon loads the data while the engine creates
 * the GPU context, the two in parallel (Sec. 4.1, Sec. 5.1); all invocations of a
 * function on a GPU share the daemon's one read-only copy (Sec. 6.2).  Here:
 *
 *   owner process : pool created with exportable = 1; sage_share_start serves the
 *                   functions given to sage_share_register on a UNIX socket;
 *   function process : sage_attach_begin (no CUDA call: it only sends the request,
 *                   and the owner starts staging at once), then its own context
 *                   (sage_pool_create), then sage_attach_end, which maps the owner's
 *                   copy and returns before the data is complete.  Invocations wait
 *                   for the owner's "complete" word exactly as for local staging.
 *
 * Each attached handle holds one reference in the owner's pool until it is
 * released, or its process exits (the socket closes); the owner stages a key
 * once however many processes attach.  The read-only copy is mapped read-write
 * in the function process; the functions here only read it.  Both processes must
 * use the same physical GPU (checked by UUID). */
typedef struct sage_share_s* sage_share;
typedef struct sage_ticket_s* sage_ticket;

typedef struct {
    int64_t connections;   /* attach requests received */
    int64_t grants;        /* requests answered with a mapping */
    int64_t rejects;       /* requests refused (unknown key, other shape, failed prepare) */
    int64_t ready;         /* "data complete" words sent */
    int64_t releases;      /* references returned (release or disconnect) */
    int64_t active;        /* attached references held now */
} sage_share_stats;

/* Serve `pool`'s functions to other processes on the UNIX socket `socket_path`
 * (created; an existing file of that name is replaced).  The pool must be
 * exportable.  SAGE_ERR_INVALID for a non-exportable pool or a path longer than
 * 107 bytes; SAGE_ERR_CUDA when the socket cannot be created. */
sage_status sage_share_start(sage_pool pool, const char* socket_path, sage_share* out);
/* Make a function attachable by key.  The descriptor (with its data sources) is
 * copied; its producer contexts and host images must stay valid until
 * sage_share_stop.  The owner prepares the key on the first attach request. */
sage_status sage_share_register(sage_share share, const sage_fn_desc* desc);
sage_status sage_share_stats_get(sage_share share, sage_share_stats* out);
/* Stop serving: closes the socket, returns every attached reference (the owner's
 * copy stays mapped in processes that still use it until they release it). */
sage_status sage_share_stop(sage_share share);

/* Send an attach request for `shape` (data sources ignored) to the owner at
 * `socket_path`.  Makes no CUDA call.  SAGE_ERR_INVALID for a bad shape or when no
 * owner listens there. */
sage_status sage_attach_begin(const char* socket_path, const sage_fn_desc* shape, sage_ticket* out);
/* Complete an attach in `pool` (consumes the ticket, also on failure): receives
 * the owner's answer, maps its copy, builds this process's workspaces and returns
 * the handle (refcount semantics as sage_prepare; a key this pool already holds is
 * shared locally).  The owner's refusal status is returned as is (SAGE_ERR_INVALID
 * for an unknown key or another shape, SAGE_ERR_NOMEM, ...); SAGE_ERR_INVALID when
 * the owner uses another GPU; SAGE_ERR_CUDA when the mapping fails;
 * SAGE_ERR_TIMEOUT when the owner does not answer within 60 s.  A staging failure
 * in the owner makes the handle sticky-failed (SAGE_ERR_STAGING). */
sage_status sage_attach_end(sage_pool pool, sage_ticket ticket, sage_fn* out);
/* Drop a ticket without completing it (closes the request; the owner returns any
 * reference it took).  Makes no CUDA call. */
sage_status sage_attach_cancel(sage_ticket ticket);

/* ---------------------------------------------------------------- SM partitions
 *
 * Functions served side by side on one GPU compete for its SMs; the paper lists
 * partitioning the SMs between functions among its lessons (Sec. 7.10).  A
 * partition splits the device's SMs into `groups` equal groups (green contexts)
 * of min_sms SMs each, rounded up to the hardware's partition granularity, or,
 * with min_sms = 0, of SMs / groups rounded down to it.  Kernels launched on a group's stream
 * run only on that group's SMs; sage_invoke* on such a stream keeps the whole
 * launch chain on it (no bottom-MLP branch stream, no CUDA graph), so every
 * kernel of the function stays inside the group.  SAGE_ERR_INVALID when the SMs
 * cannot hold the groups; SAGE_ERR_CUDA when green contexts are unavailable. */
typedef struct sage_partition_s* sage_partition;
sage_status sage_partition_create(int device, int groups, int min_sms, sage_partition* out);
int sage_partition_groups(sage_partition p);
/* Group g's stream (a cudaStream_t owned by the partition) and its SM count. */
sage_status sage_partition_stream(sage_partition p, int group, void** stream, int* sms);
/* Waits for the groups' streams, then destroys them and the green contexts;
 * SAGE_ERR_CUDA when that wait reported a device failure (destroyed anyway). */
sage_status sage_partition_destroy(sage_partition p);

#ifdef __cplusplus
}
#endif
#endif /* SAGE_H */
