/*
 * skel.h -- C ABI of libskel.so: data-parallel skeletons over smart
 * containers on one NVIDIA GB300 (sm_103a).
 *
 * Concepts (Kessler, Dastgeer, Li, "Optimized Composition: Generating
 * Efficient Code for Heterogeneous Systems from Multi-Variant Components,
 * Skeletons and Containers", 2014):
 *   - Skeletons (Sec. III): generic components derived from the higher-order
 *     functions map, reduce and scan, plus mapoverlap (SkePU), instantiated
 *     with a user function.  Here the user functions are a fixed, compiled-in
 *     set (skel_fn).
 *   - Multi-variant skeletons (Sec. III) and off-line tuned dispatch
 *     (Sec. II, "tree-based dispatch structure for fast runtime lookup"): each
 *     call is routed to one of several CUDA implementation variants, chosen by
 *     looking up the call context (skeleton, user function, element type,
 *     problem-size bucket, stencil radius, data residency) in an execution
 *     plan table built off-line by measurement.  Variants carry selectability
 *     constraints (conditional composition, Sec. II): a variant whose
 *     constraint fails for a call is never chosen.
 *   - Smart containers (Sec. IV): every non-scalar operand is a container
 *     that tracks which memory unit (host, device) holds a valid copy and
 *     copies lazily, only when the accessing unit holds no valid copy.
 *     Dependence tracking: each container remembers the stream and event of
 *     its last device write; a later access on another stream or from the
 *     host waits for it.
 *
 * Conventions for every function below:
 *   - Return value: a skel_status; SKEL_OK (0) on success, a negative code
 *     otherwise.  Nothing throws across the ABI.  On failure
 *     skel_last_error() returns a message (thread-local), and out-parameters
 *     are left unchanged.
 *   - stream: a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Skeleton calls are enqueued on it and return without waiting,
 *     except where a host result pointer is given (the call then waits for
 *     the result).
 *   - Containers are owned by the library; the caller creates and destroys
 *     them.  Memory wrapped with skel_container_wrap stays owned by the
 *     caller and must outlive the container.
 *   - Sizes are 64-bit element counts.  n = 0 is valid everywhere (reduce
 *     returns the identity, map/scan/mapoverlap do nothing).
 *   - Layout: 1D containers are contiguous; 2D containers are row-major with
 *     no padding (element (i, j) of a rows x cols container is at i*cols + j).
 *   - Element types: SKEL_F32 for all floating-point skeletons; SKEL_I32 for
 *     integer reduce and scan, whose (+) wraps modulo 2^32; SKEL_I64 for
 *     offsets of batched instances.
 */
#ifndef SKEL_H
#define SKEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct skel_container_s *skel_handle;
typedef struct skel_plan_s *skel_plan;

typedef enum {
    SKEL_F32 = 0,
    SKEL_I32 = 1,
    SKEL_I64 = 2
} skel_dtype;

typedef enum {
    SKEL_OK = 0,
    SKEL_ERR_INVALID_ARG = -1, /* bad handle, NULL pointer, aliasing not allowed */
    SKEL_ERR_SHAPE = -2,       /* operand sizes do not fit together */
    SKEL_ERR_DTYPE = -3,       /* element type not supported for this call */
    SKEL_ERR_UNSUPPORTED = -4, /* user function / option not offered by this skeleton */
    SKEL_ERR_OOM = -5,         /* allocator returned NULL */
    SKEL_ERR_CUDA = -6,        /* a CUDA runtime call failed (message has the CUDA error) */
    SKEL_ERR_TIMEOUT = -7,     /* a bounded device-side wait gave up (see skel_check_device) */
    SKEL_ERR_TABLE = -8        /* dispatch table file unreadable or malformed */
} skel_status;

/* User functions (Sec. III: the problem-specific code a skeleton is
 * parameterised with).  Which skeleton accepts which function is listed at
 * each entry point. */
typedef enum {
    SKEL_FN_ADD = 0,      /* x + y          (map, reduce/scan operator) */
    SKEL_FN_MUL = 1,      /* x * y          (map, mapreduce map: dot product) */
    SKEL_FN_MAX = 2,      /* max(x, y)      (map, reduce operator) */
    SKEL_FN_AXPY = 3,     /* a * x + y      (map; params[0] = a) */
    SKEL_FN_TANH = 4,     /* tanh(x)        (map) */
    SKEL_FN_SQ = 5,       /* x * x          (map, mapreduce map: sum of squares) */
    SKEL_FN_SCALE = 6,    /* a * x          (map; params[0] = a) */
    SKEL_FN_SUB = 7,      /* x - y          (map) */
    SKEL_FN_COPY = 8,     /* x              (map) */
    SKEL_FN_STENCIL5 = 9, /* 2D 5-point cross (mapoverlap), radius 1 */
    SKEL_FN_STENCIL9 = 10,/* 2D 3x3 box (mapoverlap), radius 1 */
    SKEL_FN_STENCIL1D = 11,/* 1D weighted window of radius r <= 16 (mapoverlap) */
    SKEL_FN_GATHER = 12,  /* out[i] = A[clamp(idx[i], 0, m-1)] (maparray) */
    SKEL_FN_ROWDOT = 13,  /* out[i] = sum_k A[k] * M[i, k]     (maparray) */
    SKEL_FN_COULOMB = 14  /* potential of point charges on a grid (maparray over a grid) */
} skel_fn;

typedef enum {
    SKEL_CLAMP = 0,    /* reads outside the range take the nearest edge value */
    SKEL_ZERO = 1,     /* reads outside the range are 0 */
    SKEL_PERIODIC = 2  /* reads wrap around */
} skel_boundary;

typedef enum { SKEL_READ = 1, SKEL_WRITE = 2, SKEL_READWRITE = 3 } skel_access;

/* Memory units of the coherence protocol (bits of a valid set). */
typedef enum { SKEL_UNIT_HOST = 1, SKEL_UNIT_DEVICE = 2 } skel_unit;

/* Skeletons, as keys of the dispatch table and of skel_force_variant. */
typedef enum {
    SKEL_SK_MAP = 0,
    SKEL_SK_REDUCE = 1,
    SKEL_SK_MAPREDUCE = 2,
    SKEL_SK_SCAN = 3,
    SKEL_SK_MAPOVERLAP1D = 4,
    SKEL_SK_MAPOVERLAP2D = 5,
    SKEL_SK_MAPARRAY = 6,
    SKEL_SK_BATCHED = 7,
    SKEL_SK_CHAIN2D = 8,   /* a chain of 2D MapOverlap calls (skel_mapoverlap_chain) */
    SKEL_SK_EDGE = 9,      /* host edge of Map / Reduce / MapReduce calls on host-only inputs */
    SKEL_SK_COMPOSE = 10,  /* Map -> MapOverlap -> MapReduce chain (skel_compose_map_stencil_sumsq) */
    SKEL_SK_COUNT = 11
} skel_skeleton;

/* ------------------------------------------------------------ library --- */

/* Version string of the library (static storage). */
const char *skel_version(void);

/* Message of the last failed call on this thread ("" if none).  The pointer
 * stays valid until the next call on this thread. */
const char *skel_last_error(void);

/* Device memory allocator used for container storage and kernel scratch.
 * alloc(bytes, stream, ctx) returns device memory usable on `stream` or NULL;
 * free(ptr, stream, ctx) releases it (stream-ordered).  Passing NULL for
 * alloc restores the built-in allocator (cudaMallocFromPoolAsync on the library's own pool / cudaFreeAsync).
 * Containers and scratch already allocated keep the allocator they were
 * allocated with.  Not thread-safe against concurrent skeleton calls. */
int skel_set_allocator(void *(*alloc)(size_t bytes, void *stream, void *ctx),
                       void (*free_fn)(void *ptr, void *stream, void *ctx), void *ctx);

/* Releases the cached scratch memory and result slots of every stream, and
 * returns the unused memory of the built-in allocator's pools (the library
 * keeps its own pool per device, which holds freed memory for later calls).
 * Containers are not touched.  Waits for the streams that used them. */
int skel_release_cached(void);

/* Number of CUDA kernels the library has launched in this process (all
 * threads, all devices); a skeleton call launches one to four. */
int64_t skel_launch_count(void);

/* ------------------------------------------------ smart containers (IV) --- */

/* Creates a container of `ndim` (1 or 2) dimensions; shape[0] (and shape[1]
 * for 2D: rows, cols) >= 0.  Storage is allocated lazily by the library on
 * first access by each unit (device memory through the allocator, host memory
 * pinned).  No unit holds a valid copy yet (contents undefined). */
int skel_container_create(skel_dtype dtype, int ndim, const int64_t *shape, skel_handle *out);

/* Creates a container over caller-owned memory.  host_ptr and/or dev_ptr may
 * be NULL (the library then allocates that side lazily).  valid_units (bits
 * of skel_unit) states which of the given pointers hold the data now.  The
 * caller keeps ownership and must keep the memory alive until
 * skel_container_destroy. */
int skel_container_wrap(skel_dtype dtype, int ndim, const int64_t *shape, void *host_ptr,
                        void *dev_ptr, int valid_units, skel_handle *out);

/* A view of `count` elements of `parent` starting at element `offset`,
 * reshaped to ndim/shape (product of shape == count).  The view shares the
 * parent's storage and coherence state (whole-operand granularity: a write
 * through a view invalidates the other unit's copy of the whole parent).
 * Destroy views before their parent. */
int skel_container_view(skel_handle parent, int64_t offset, int ndim, const int64_t *shape,
                        skel_handle *out);

/* Host access (Sec. IV lazy copying): if mode reads and the host copy is not
 * valid, copies device -> host on `stream` and waits for it; otherwise waits
 * for the last device write.  mode = SKEL_WRITE / SKEL_READWRITE leaves the
 * host as the only valid copy (the caller then writes through the pointer).
 * Returns the host address of the container's first element in *ptr. */
int skel_container_host_ptr(skel_handle h, int mode, void *stream, void **ptr);

/* Device access: if mode reads and the device copy is not valid, enqueues a
 * host -> device copy on `stream`; makes `stream` wait for the last device
 * write if it was made on another stream.  A writing mode leaves the device
 * as the only valid copy.  Returns the device address in *ptr. */
int skel_container_device_ptr(skel_handle h, int mode, void *stream, void **ptr);

/* Declares that the caller wrote the given units' copies directly (through a
 * wrapped pointer): the valid set becomes exactly `units`. */
int skel_container_mark(skel_handle h, int units);

/* Starts, without waiting, the copy that makes `unit` (SKEL_UNIT_HOST or
 * SKEL_UNIT_DEVICE) hold a valid copy: the lazy copy of Sec. IV issued
 * early, so that it overlaps other work.  Enqueued on `stream` after the
 * container's last device use (on whatever stream that was); later accesses
 * order after it (a host access waits for it).  Nothing is copied when
 * `unit` is already valid or no unit is.  A host copy is allocated (pinned)
 * if the container has none. */
int skel_container_prefetch(skel_handle h, int unit, void *stream);

/* Shape and state: dtype, ndim, shape[2] (shape[1] = 1 for 1D), bits of the
 * units that currently hold a valid copy. */
int skel_container_info(skel_handle h, int *dtype, int *ndim, int64_t *shape, int *valid_units);

/* Transfer statistics since creation (shared with views): counts and bytes
 * of host->device and device->host copies. */
int skel_container_stats(skel_handle h, int64_t *h2d_count, int64_t *d2h_count,
                         int64_t *h2d_bytes, int64_t *d2h_bytes);

/* Destroys the container; frees library-owned storage (stream-ordered on the
 * stream of its last device use). */
int skel_container_destroy(skel_handle h);

/* The protocol step itself, a pure host function: given the valid set,
 * the accessing unit and the access mode, returns the new valid set and the
 * transfer it needs (0 none, 1 host->device, 2 device->host).  Every
 * container access goes through this function. */
int skel_coherence_step(int valid_units, int unit, int mode, int *new_valid, int *transfer);

/* ------------------------------------------------ skeleton calls (III) --- */

/* Map: out[i] = f(in0[i], in1[i]; params) for i < n.
 * fn: ADD, SUB, MUL, MAX (2 inputs); AXPY (2 inputs, params[0] = a);
 *     TANH, SQ, COPY (1 input); SCALE (1 input, params[0] = a).
 * All operands SKEL_F32 with the same element count (shapes may differ).
 * out may be the same container as an input, or another container over the
 * same device memory (in place: every variant then runs without the
 * read-only load path).  An output that shares only part of an input's
 * bytes (a shifted view, or a wrapped pointer into it) returns
 * SKEL_ERR_INVALID_ARG before any copy or launch. */
int skel_map(skel_fn fn, const double *params, int nparams, const skel_handle *ins, int nin,
             skel_handle out, void *stream);

/* Reduce: r = in[0] (+) in[1] (+) ... with op ADD or MAX.
 * F32: ADD is float32 arithmetic in a fixed, size-determined order
 *      (deterministic); identity 0 (ADD) and -inf (MAX).
 * I32: ADD wraps modulo 2^32; identity 0 (ADD) and INT32_MIN (MAX).
 * result_host (may be NULL): receives the result (4 bytes); the call then
 * waits.  result_dev (may be NULL): a 1-element container of the same dtype
 * that receives the result on the device. */
int skel_reduce(skel_fn op, skel_handle in, void *result_host, skel_handle result_dev,
                void *stream);

/* MapReduce: r = (+)_i f(in0[i], in1[i]) with reduce op ADD and map fn MUL
 * (dot product, 2 inputs) or SQ (sum of squares, 1 input).  F32 only.
 * Results as for skel_reduce. */
int skel_mapreduce(skel_fn map_fn, skel_fn red_op, const skel_handle *ins, int nin,
                   void *result_host, skel_handle result_dev, void *stream);

/* Scan with op ADD: inclusive out[i] = in[0] + ... + in[i]; exclusive
 * out[0] = 0, out[i] = in[0] + ... + in[i-1].  A 2D container is scanned
 * along each row independently.  I32 (wraps modulo 2^32) or F32 (float32
 * element arithmetic; the carry between tiles is kept in float64).
 * out must not be the same container as in. */
int skel_scan(skel_fn op, int inclusive, skel_handle in, skel_handle out, void *stream);

/* Allocation-free scan.  The paper has no counterpart to this entry point; it
 * exists for callers that cannot allocate device memory: a host that hands
 * the library a fixed memory budget and owns every allocation itself, or a
 * latency-critical host path that must not take an allocator's lock or risk
 * the device-wide synchronisation that cudaMalloc and cudaFree can cause.
 * It computes what skel_scan computes for a 1D operand (op ADD, inclusive or
 * exclusive, dtype SKEL_I32 wrapping modulo 2^32 or SKEL_F32 with a float64
 * carry), but on raw device pointers and without containers: `in` and `out`
 * are caller-owned device arrays of n elements of `dtype` that must not
 * overlap.  The call allocates nothing: its scratch (a tile counter and the
 * look-back words) is a static device array of 512 KiB + 256 bytes inside
 * libskel.so, which every GPU that loads the library holds until the process
 * exits.  n must be <= SKEL_SCAN_NOALLOC_MAX_N (2^27, the array's capacity);
 * larger n returns SKEL_ERR_SHAPE without launching.  The first call on each
 * device looks up the array's device address and clears it (stream-ordered
 * on `stream`); make that first call before any stream capture.  The array
 * also holds the tag that marks which call wrote a look-back word: the
 * kernel reads it, and its last block to finish advances it (clearing the
 * words every 255 calls), so consecutive calls need nothing from the host
 * besides the address.  Every call shares the array and each leaves it ready
 * for the next, so calls that overlap on the GPU (on two streams at once, or
 * from two threads) race on it and must be serialised by the caller.  A
 * bounded look-back wait that gives up (skel_set_debug key 2) is recorded in
 * the array and reported, and cleared, by the next skel_check_device on this
 * device, as for skel_scan.  Enqueued on `stream`; returns without waiting. */
#define SKEL_SCAN_NOALLOC_MAX_N ((int64_t)1 << 27)
int skel_scan_noalloc(skel_fn op, int inclusive, skel_dtype dtype, const void *in, void *out, int64_t n,
                      void *stream);

/* MapOverlap (SkePU mapoverlap, Sec. III): each output reads a fixed
 * neighbourhood of its input position.
 *   1D (in is 1D), fn = STENCIL1D: out[i] = sum_{k=-r..r} w[k+r] * in[b(i+k)],
 *     radius 0 <= r <= 16, nweights = 2r+1 (weights NULL: binomial weights
 *     C(2r, k) / 4^r).
 *   2D (in is 2D), fn = STENCIL5 or STENCIL9, radius must be 1:
 *     out[i,j] = sum_{di,dj} w[di,dj] * in[b(i+di), b(j+dj)] with w given as
 *     9 values row-major over (di, dj) in [-1,1]^2 (STENCIL5 reads only the
 *     centre and the 4 edge-adjacent entries).  weights NULL: STENCIL5 =
 *     centre 1/2, N/S/W/E 1/8; STENCIL9 = [1 2 1]^T [1 2 1] / 16.
 *   b: the boundary map, applied to each axis.  F32 only.
 * out must not be the same container as in. */
int skel_mapoverlap(skel_fn fn, int radius, const float *weights, int nweights,
                    skel_boundary boundary, skel_handle in, skel_handle out, void *stream);

/* A chain of `steps` 2D MapOverlap calls, each reading the previous one's
 * output: out = S^steps(in) with S the stencil of skel_mapoverlap (same fn,
 * weights and boundary; radius 1).  The composition is one call so that its
 * implementation is chosen for the chain, not call by call (Sec. II: the
 * global composition problem; Sec. IV: intermediate results stay on the
 * device).  Variants: per_call (steps single MapOverlap calls, each
 * dispatched as skel_mapoverlap would be) and time_blocked (tile = steps per
 * pass, 1..8: a block stages its tile with that many halo cells and applies
 * the passes' steps in shared memory; CLAMP and ZERO only), which gives the
 * per-call result bit for bit.  in, tmp and out are 2D F32 of one shape and
 * pairwise distinct; tmp holds intermediate steps (NULL allowed when steps
 * == 1 or when a single time-blocked pass covers all steps; a variant that
 * needs it then refuses and the call falls back).  in is not modified.
 * steps >= 1.  Enqueued on `stream`. */
int skel_mapoverlap_chain(skel_fn fn, const float *weights, int nweights, skel_boundary boundary, int steps,
                          skel_handle in, skel_handle tmp, skel_handle out, void *stream);

/* The chain Map -> MapOverlap -> MapReduce as one call (Sec. II: the
 * implementation is selected for the composition, not call by call):
 *   result = sum_{i,j} (S t)[i,j]^2,   t = map_fn(in)
 * map_fn: TANH, SQ, SCALE (params[0] = a, nparams >= 1) or COPY; S: the 2D
 * stencil of skel_mapoverlap (stencil = STENCIL5 or STENCIL9, radius 1,
 * weights NULL or 9 values, boundary on t: outside a ZERO boundary t reads
 * 0).  in: 2D F32.  The result (F32) goes to result_host (the call then
 * waits) and/or to result_dev (a 1-element F32 container); at least one.
 * Table key (SKEL_SK_COMPOSE, stencil, F32, n, radius 1, residency).
 * Variants: per_call (the Map, MapOverlap and MapReduce calls, each
 * dispatched as usual, through two n-element temporaries: 20 bytes of HBM
 * traffic per point) and fused (tile 0..2: 32 << tile rows per block; one
 * pass reading in once, 4 bytes per point, then one Reduce of the block
 * partials; needs 16-byte aligned rows, cols % 4 == 0).  Both compute every
 * stencil output with the same float32 operations; the sums differ in
 * order only.  n = 0 gives 0. */
int skel_compose_map_stencil_sumsq(skel_fn map_fn, const double *params, int nparams, skel_fn stencil,
                                   const float *weights, int nweights, skel_boundary boundary, skel_handle in,
                                   void *result_host, skel_handle result_dev, void *stream);

/* MapArray: out[i] = f(A, B[i]) with A read whole (random access) and B per
 * element.  The paper does not define MapArray; the reading used is:
 *   GATHER: A 1D F32 of length m >= 1, B 1D I32 of length n,
 *           out 1D F32 of length n, out[i] = A[clamp(B[i], 0, m-1)].
 *   ROWDOT: A 1D F32 of length m, B 2D F32 of shape (n, m),
 *           out 1D F32 of length n, out[i] = sum_k A[k] * B[i, k]. */
int skel_maparray(skel_fn fn, skel_handle whole, skel_handle elem, skel_handle out, void *stream);

/* MapArray whose element is its own position on a regular grid: the
 * Coulombic potential grid that Sec. III runs with SkePU skeletons (Fig. 2).
 *   fn = COULOMB: whole = atoms, 2D F32 of shape (m, 4), row k = (x_k, y_k,
 *   z_k, q_k), 16-byte aligned; out = 2D F32 (rows, cols), out[i, j] at the
 *   point (j*h, i*h, z0):
 *     out[i, j] = sum_k q_k / sqrt((j*h - x_k)^2 + (i*h - y_k)^2 + (z0 - z_k)^2)
 *   params = {h, z0} (nparams = 2), h > 0.  A point that coincides with an
 *   atom gets an infinite term (as the definition does); so does one whose
 *   squared distance is below 2^-126 (float32 subnormal, flushed to 0).  Each
 *   term uses the hardware reciprocal square root (PTX rsqrt.approx, relative
 *   error within 2^-22.9); terms are accumulated with compensation, so
 *   |out - exact| stays within a few units of 2^-24 * sum_k |q_k| / r_k.
 *   m = 0 gives zeros.
 * The library reads the atoms and writes out on the device (lazy copies as
 * for every skeleton); enqueued on `stream`.  Errors: SKEL_ERR_DTYPE /
 * SKEL_ERR_SHAPE for other types or shapes, SKEL_ERR_INVALID_ARG for h <= 0,
 * wrong nparams, a misaligned atom array or out aliasing the atoms. */
int skel_maparray_grid(skel_fn fn, skel_handle whole, skel_handle out, const double *params, int nparams,
                       void *stream);

/* Batched instances: B independent float32 instances laid end to end in
 * `values`; instance b is values[offsets[b] .. offsets[b+1]) with offsets an
 * I64 container of B+1 non-decreasing entries, offsets[0] = 0,
 * offsets[B] = length of values.  One persistent launch computes, for every
 * instance, results[b] = (+)_i f(x_i) (map_fn SQ, red_op ADD; results F32 of
 * length B, may be NULL) and the scan (scan_op ADD, inclusive or exclusive)
 * of the instance into scan_out (F32, same length as values, may be NULL). */
int skel_batched(skel_fn map_fn, skel_fn red_op, skel_fn scan_op, int inclusive,
                 skel_handle values, skel_handle offsets, skel_handle results,
                 skel_handle scan_out, void *stream);

/* The same batched call captured once into a CUDA graph: plan_create
 * allocates the scratch memory, captures the launch sequence and
 * instantiates it; plan_launch replays the graph on `stream` (the containers'
 * device copies must be valid and must keep their device addresses).  The
 * plan holds references to the containers' device memory, not to the
 * handles' coherence state: a replay marks nothing. */
int skel_batched_plan_create(skel_fn map_fn, skel_fn red_op, skel_fn scan_op, int inclusive,
                             skel_handle values, skel_handle offsets, skel_handle results,
                             skel_handle scan_out, void *stream, skel_plan *plan);
int skel_plan_launch(skel_plan plan, void *stream);
int skel_plan_destroy(skel_plan plan);

/* ---------------------------------------------- backward (adjoint) calls --- */

/* Adjoint of skel_map: gins[k][i] = gout[i] * d f / d in_k (in0[i], in1[i]).
 * Same functions and operand rules as skel_map; gins has nin entries, an
 * entry may be NULL when that gradient is not wanted.  For TANH, ins[0] may
 * be the saved forward OUTPUT instead of the input when params = {1.0}
 * (nparams = 1): then d tanh = 1 - out^2 without recomputing tanh. */
int skel_map_bwd(skel_fn fn, const double *params, int nparams, const skel_handle *ins, int nin,
                 skel_handle gout, skel_handle *gins, void *stream);

/* skel_map_bwd when the map's output feeds several calls (a composition of
 * calls, Sec. II): the upstream gradient is gouts[0] + gouts[1] (ngout 1 or
 * 2, same length and type), added inside the adjoint's own pass instead of
 * by a separate Map (ADD) call.  Otherwise as skel_map_bwd. */
int skel_map_bwd_sum(skel_fn fn, const double *params, int nparams, const skel_handle *ins, int nin,
                     const skel_handle *gouts, int ngout, skel_handle *gins, void *stream);

/* Adjoint of skel_reduce with ADD: gin[i] = gr for every i (a broadcast);
 * gr is a 1-element F32 container (device) or, if gr is NULL, *gr_host. */
int skel_reduce_bwd(skel_fn op, skel_handle gr, const float *gr_host, skel_handle gin,
                    void *stream);

/* Adjoint of skel_mapreduce with ADD: gins[k][i] = gr * d f / d in_k.
 * gr as in skel_reduce_bwd. */
int skel_mapreduce_bwd(skel_fn map_fn, skel_fn red_op, const skel_handle *ins, int nin,
                       skel_handle gr, const float *gr_host, skel_handle *gins, void *stream);

/* Adjoint of skel_scan with ADD: the reverse scan.  inclusive:
 * gin[j] = sum_{i>=j} gout[i]; exclusive: sum_{i>j} gout[i].  2D: per row.
 * F32 only. */
int skel_scan_bwd(skel_fn op, int inclusive, skel_handle gout, skel_handle gin, void *stream);

/* Adjoint of skel_mapoverlap: gin = S^T gout, the transposed stencil.  With
 * CLAMP, taps that the forward pass clamped onto an edge element fold their
 * weight back onto that edge element; ZERO and PERIODIC transpose to the
 * mirrored stencil.  Same arguments as skel_mapoverlap. */
int skel_mapoverlap_bwd(skel_fn fn, int radius, const float *weights, int nweights,
                        skel_boundary boundary, skel_handle gout, skel_handle gin, void *stream);

/* ------------------------------------------- variant dispatch (II, III) --- */

/* Loads an execution-plan table (text, one entry per line; see the table
 * writer of the autotuner):
 *   skeleton fn dtype bucket radius residency variant block ept tile
 * bucket = floor(log2(n) / 2) (n elements; n = 0 uses bucket 0); variant -1
 * records that the built-in default is the best choice for that key.  Entries
 * replace the built-in defaults for their key; a call whose key has no entry
 * uses the entry of the nearest lower tuned bucket of the same (skeleton, fn,
 * dtype, radius, residency), else the nearest higher one, else the built-in
 * default.  path NULL clears the table (built-in defaults only). */
int skel_load_dispatch_table(const char *path);

/* Adds or replaces one table entry (same fields as a table line). */
int skel_dispatch_set(int skeleton, int fn, int dtype, int bucket, int radius, int residency,
                      int variant, int block, int ept, int tile);

/* Number of entries in the table. */
int skel_dispatch_size(void);

/* Forces every call of `skeleton` onto one variant and launch shape
 * (block, ept, tile; 0 = the variant's own default) regardless of the table;
 * variant = -1 removes the force.  A forced variant whose selectability
 * constraint fails for a call makes that call return SKEL_ERR_UNSUPPORTED. */
int skel_force_variant(int skeleton, int variant, int block, int ept, int tile);

/* Variant, block, ept and tile the last call of `skeleton` ran with on this
 * thread (all -1 before the first call). */
int skel_last_variant(int skeleton, int *variant, int *block, int *ept, int *tile);

/* The host edge (SKEL_SK_EDGE; Sec. IV lazy copying, keyed by residency).
 * A Map, Reduce or MapReduce call with an input whose valid copy is only in
 * host memory first chooses, from the entries of skeleton SKEL_SK_EDGE
 * (fn = the calling skeleton: SKEL_SK_MAP, SKEL_SK_REDUCE or
 * SKEL_SK_MAPREDUCE; residency 1), how those bytes cross the host link:
 *   variant 0 copy:    the whole lazy copy, then the call (the default);
 *   variant 1 chunked: the copy in chunks of 8 MiB << (2 * tile) bytes
 *                      (tile 0..3) on a library-owned copy stream, each
 *                      chunk's part of the call started on `stream` as soon
 *                      as the chunk has landed; afterwards the input is valid
 *                      on both units, as after the whole copy.  Needs inputs
 *                      that cover their whole storage (no views);
 *   variant 2 direct:  the kernels read the host copy in place over the link;
 *                      no device copy is made and the input stays valid only
 *                      on the host.  Needs pinned host memory (cudaMallocHost,
 *                      cudaHostAlloc or registered); the caller must not
 *                      write the host copy until `stream` has finished the
 *                      call, as for an asynchronous copy.
 * Neither 1 nor 2 applies when the output shares storage with a host-only
 * input.  Second touch: an input that has already been read in place (2)
 * since its host copy was last written (host write access, or
 * skel_container_mark) is being reused, so a table choice of 2 becomes 0 for
 * it and later calls find it on the device.  A variant that does not apply falls back to 0 (or, when forced,
 * makes the call return SKEL_ERR_UNSUPPORTED).  skel_last_variant(SKEL_SK_EDGE)
 * reports the choice of the last such call. */

/* Number of variants of a skeleton and the name of variant v (static). */
int skel_variant_count(int skeleton);
const char *skel_variant_name(int skeleton, int variant);

/* ---------------------------------------------------- device status ---- */

/* Waits for `stream` and reports device-side failures of the calls made on
 * it since the last check (and of skel_scan_noalloc calls on the current
 * device, whose status sits in its static array): SKEL_ERR_TIMEOUT if a
 * bounded wait (the scan's look-back over predecessor tiles, a TMA copy)
 * gave up, SKEL_ERR_INVALID_ARG
 * if a batched call found its device-resident offsets invalid (that call
 * computed nothing), SKEL_OK otherwise.  Clears the recorded status. */
int skel_check_device(void *stream);

/* Test hooks for failure detection without a GPU fault.  key 1: the
 * look-back tile with this index (value; -1 = off) never publishes its
 * result, so its successors' bounded waits run out (the look-back scan
 * variants and the re-reading batched variant).  key 2: the bounded wait's
 * limit in microseconds (default 2,000,000). */
int skel_set_debug(int key, int64_t value);

/* ------------------------------------------------ measurement probes --- */

/* Enqueues `count` launches of an empty kernel on `stream`, back to back.
 * Timed with events around them, they give this GPU's launch floor: the
 * least time a call made of k dependent launches can take (the bound of a
 * small, latency-bound call such as the MapReduce dot product at n = 2^20).
 * Returns without waiting. */
int skel_probe_empty_launches(int count, void *stream);

/* Enqueues about `reads` random 4-byte reads from `table` (device memory, m
 * floats, m a power of two <= 2^31; it stays in L2 when m * 4 bytes is well
 * below the L2's size) over one wave of blocks, with indices from a
 * per-thread generator in registers and no output stream; `sink` (one
 * device float) is never written in practice.  *reads_made receives the
 * number of reads the launch makes (rounded up to whole batches).  Timed with
 * events, reads_made / time is the random-sector rate that bounds MapArray's
 * gather, whose reads of A have the same pattern.  Returns without waiting. */
int skel_probe_l2_random(const float *table, int64_t m, int64_t reads, float *sink, int64_t *reads_made,
                         void *stream);

/* The host cost of a skeleton call against a bare launch of its kernel
 * (Sec. IV: the smart containers' overhead).  Creates three float32
 * containers of n elements (device-valid), then times on the host, with a
 * steady clock, `calls` skel_map(AXPY) calls (argument checks, table lookup,
 * the coherence steps of three operands, the launch) and `calls` launches of
 * the same kernel variant with the same arguments and no container or table
 * work.  *us_call and *us_launch receive microseconds per call.  Synchronises
 * `stream`; destroys the containers.  With calls kept below the device's
 * launch queue depth (a few hundred) neither loop waits for the GPU. */
int skel_probe_call_overhead(int calls, int64_t n, double *us_call, double *us_launch, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SKEL_H */
