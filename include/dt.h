/*
 * dt.h -- C ABI of the GB300 sample-based divide-and-conquer Delaunay
 * triangulation (Funke, Sanders, Winkler: "Load-Balancing for Parallel
 * Delaunay Triangulations").
 *
 * What is computed (Sec. 2.1): DT(P) for a point set P in R^2 or R^3 -- the
 * triangulation of conv(P) whose vertex set is P and in which no point lies
 * inside the circumsphere of any simplex.  Ties (cocircular / cospherical
 * subsets) are resolved by a symbolic perturbation of the lifting map that
 * ranks points by their input index, so the result is unique for every
 * duplicate-free input and does not depend on k, the sample or the seed.
 *
 * How (Alg. 1 with the divide step of Alg. 2): sample eta points, triangulate
 * them, partition the sample's Delaunay graph into k balanced blocks, label
 * every point with the block of its nearest sample point, triangulate the k
 * partitions independently, detect border simplices whose circumsphere may
 * reach another partition, triangulate the border vertices, and merge with
 * hash-table lookups.  Every step runs in CUDA kernels on one GPU.
 *
 * Conventions for every entry point
 *   - Return value: 0 on success, a negative DT_E_* code otherwise.  No call
 *     aborts the process; after an error the context stays usable and
 *     dt_last_error() describes the failure.
 *   - Pointers marked "host or device" may point to host memory or to device
 *     memory of the context's GPU; the library detects which.
 *   - Points are float64, row-major (n x dim).  Indices are 0-based input
 *     order.  Simplices are returned as int32 vertex indices, each tuple
 *     sorted ascending, the whole array sorted lexicographically; only
 *     finite simplices are returned.
 *   - The library owns its results until the next dt_triangulate on the same
 *     context or dt_destroy.  The caller owns every buffer it passes.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef GB300_DT_H
#define GB300_DT_H

#include <stdint.h>

#if defined(__GNUC__)
#define DT_API __attribute__((visibility("default")))
#else
#define DT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define DT_OK 0
#define DT_E_ARG (-1)        /* invalid argument (null, dim, n, k, frac, non-finite) */
#define DT_E_DUPLICATE (-2)  /* two input points coincide exactly */
#define DT_E_DEGENERATE (-3) /* all points lie on one line (2D) or plane (3D) */
#define DT_E_NOMEM (-4)      /* device allocation failed or budget exceeded */
#define DT_E_TIMEOUT (-5)    /* a device loop hit its iteration limit */
#define DT_E_OVERFLOW (-6)   /* an internal arena or table ran out of room */
#define DT_E_CUDA (-7)       /* a CUDA runtime call failed */
#define DT_E_RANGE (-8)      /* coordinates span too many binary orders of magnitude
                                for the exact fallback (> ~200 bits between the
                                largest coordinate difference and the finest bit) */
#define DT_E_INTERNAL (-9)   /* consistency check failed (a bug) */

/* Divide strategies. */
#define DT_DIVIDE_SAMPLE 0   /* Alg. 2: sample DT + graph partition + nearest-sample labels */
#define DT_DIVIDE_KD 1       /* Sec. 2.3: recursive median split, cyclic dimension */

/* Border-detection primitives (Sec. 3.2). */
#define DT_PRIM_GRID 0       /* occupied uniform-grid cells with a coarse-to-fine hierarchy */
#define DT_PRIM_BBOX 1       /* one axis-aligned bounding box per partition */
#define DT_PRIM_POINTS 2     /* the points themselves: a simplex is a border simplex when a point
                                of another partition lies in its (slightly inflated) circumsphere;
                                the grid serves as the index (Sec. 3.2, the exact primitive) */

/* Initial blocks of the sample partitioner, refined by label propagation. */
#define DT_INIT_AUTO 0       /* the default (DT_INIT_KD: lower cut weight and c_v than Hilbert runs
                                on the uniform and clustered workloads) */
#define DT_INIT_HILBERT 1    /* k equal ranges of the sample in Hilbert-curve order */
#define DT_INIT_KD 2         /* the kd median split of the sample (the cuts of DT_DIVIDE_KD) */

/* Partitioners of the sample graph (stand-ins for KaHIP, Sec. 4.3). */
#define DT_PART_LP 0         /* the initial blocks refined by lp_rounds rounds of size-constrained label
                                propagation on the sample graph */
#define DT_PART_MULTILEVEL 1 /* multilevel: heavy-edge matchings inside the initial blocks coarsen the
                                graph level by level, then label propagation with vertex weights refines
                                every level from the coarsest down, lp_rounds rounds on the sample graph
                                and max(1, lp_rounds / 2) on each coarse level (a coarse move moves a
                                whole cluster of sample points) */

/* Edge weights of the sample graph (Table 1). */
#define DT_WEIGHT_LOG 0
#define DT_WEIGHT_CONSTANT 1
#define DT_WEIGHT_INVERSE 2
#define DT_WEIGHT_LINEAR 3

typedef struct dt_config {
  int divide;            /* DT_DIVIDE_*; default DT_DIVIDE_SAMPLE */
  int primitive;         /* DT_PRIM_*; default DT_PRIM_GRID */
  int weight;            /* DT_WEIGHT_*; default DT_WEIGHT_LOG (Sec. 4.4) */
  int lp_rounds;         /* label-propagation rounds of the partitioner; default 16 */
  double epsilon;        /* partition imbalance, |V_i| <= (1+eps) ceil(|V|/k); default 0.05 */
  double grid_cell;      /* c_G: grid cell edge in units of the mean point spacing; default 1 */
  uint64_t seed;         /* sample seed; default 1 */
  int base_threshold;    /* N of Alg. 1: run k = 1 when n / k < N; default 2048 */
  int validate;          /* 1: certify the result after the merge (the checks of dt_validate);
                            a failed certificate returns DT_E_INTERNAL */
  int cavity_cap;        /* initial per-insertion cavity capacity (simplices); 0 = automatic */
  int profile;           /* 1: time the insertion kernels with CUDA events (dt_get_kernel_profile) */
  int neighbors;         /* 1: run the neighbourhood update inside dt_triangulate (otherwise it runs
                            on the first dt_get_neighbors call) */
  int first_batch;       /* points per instance in the first insertion batch (BRIO); 0 = automatic (32) */
  int brio_growth;       /* BRIO batch growth x 100: each batch has about (growth - 1) times the points
                            inserted before it; 0 = automatic (150) */
  int small_rounds;      /* rounds with at most this many active points run inside one thread block
                            (no launches between their phases); 0 or -1 = never (the default: on
                            GB300 the per-round latency is the phases' memory chains, not the
                            launches, so the graph of separate kernels is as fast or faster) */
  int brio_drain;        /* the next BRIO batch is activated when the active set has drained to
                            1 / brio_drain of the last batch; 0 = automatic (8) */
  int partition_init;    /* DT_INIT_*: initial blocks of the sample partitioner */
  int recursive;         /* 1: recursive bisection (Sec. 3.1): the divide applied log2 k times with
                            k' = 2 (a fresh sample per node, or the kd median split) and k - 1 merges,
                            batched level by level; k must be a power of two */
  int active_ratio;      /* continuous activation: before every insertion round further BRIO levels are
                            activated while the active set holds fewer than active_ratio / 100 x the
                            points inserted so far (and at least first_batch per instance); 0 = the
                            drain rule of brio_drain */
  int nominate_rings;    /* a nominee must hold the strongest pick of this round within this many
                            neighbour rings of its located simplex (1 or 2); 0 = automatic (1) */
  int partitioner;       /* DT_PART_*: the partitioner of the sample graph; default DT_PART_LP */
  int round_limit;       /* insertion rounds of one engine run before it stops with DT_E_TIMEOUT;
                            0 = 400,000 */
  int walk_limit;        /* steps of one point-location walk before DT_E_TIMEOUT; 0 = 65,536 */
  int arena_factor;      /* simplex slots per point of the insertion arena (dead slots are not reused,
                            so a 3D run needs about 27); an arena that overflows is doubled and the run
                            repeated, three times at most, then the call fails with DT_E_OVERFLOW;
                            0 = automatic (36 in 3D, 8 in 2D) */
  int cavity_blocks;     /* thread blocks per SM of the region-growth and insertion kernels (128 threads,
                            one warp per nominee; the kernels loop over the nominees); 0 = automatic (16) */
  int cavity_occupancy;  /* resident blocks per SM the region-growth kernel is compiled for: 8, 12 or 16
                            (registers per thread capped at 64, 40, 32); 0 = automatic (8) */
  int cavity_group;      /* lanes of the region-growth kernel per nominee: 32 (one warp, 8 region
                            simplices per step in 3D) or 16 (two nominees per warp, 4 per step);
                            0 = automatic (32) */
} dt_config;

typedef struct dt_stats {
  int64_t n;             /* input points */
  int64_t simplices;     /* finite simplices in the result */
  int32_t k;             /* partitions used (1 when the base case ran) */
  int32_t dim;
  int64_t eta;           /* sample size */
  int64_t border_vertices;   /* |vertices(B)| */
  int64_t border_simplices;  /* |B| */
  int64_t border_dt_simplices; /* |T_B| (finite) */
  double imbalance;      /* max_i p_i / (n/k) - 1 (Sec. 4.6) */
  double cv;             /* coefficient of variation of partition sizes, k-1 denominator */
  double o_dt;           /* overtriangulation factor (n + eta + |vertices(B)|) / n */
  int64_t cut_weight;    /* weight of sample-graph edges cut by the partition */
  int32_t rounds_max;    /* insertion rounds of the slowest triangulation */
  int32_t exact_calls;   /* exact-arithmetic fallbacks taken (saturating) */
  double ms_total;       /* device time of the whole call, ms */
  double ms_phase[8];    /* sample+graph, partition+label+scatter, partial DTs, border,
                            border DT, merge, canonicalise, neighbourhood update + validation */
  int64_t partition_size_max;
  int64_t partition_size_min;
  int64_t launches;      /* CUDA kernels this call launched */
  int64_t hull_facets;   /* facets of the convex hull (when neighbours were computed) */
  int32_t validated;     /* 1 when the certificate ran and passed */
  int32_t reserved_i;
} dt_stats;

/* Result of a certificate run (dt_validate, dt_config.validate).  The
 * rows are DT(P) under the perturbation rule exactly when violations == 0:
 * every simplex is non-flat, every facet lies in one or two simplices, the
 * two simplices on an interior facet lie on opposite sides of it and each
 * one's apex is outside the other's perturbed circumsphere (Sec. 2.1, the
 * Delaunay lemma), the boundary is locally convex at every hull ridge,
 * every point is a vertex, and the Euler characteristic is 1. */
typedef struct dt_validation {
  int64_t simplices;       /* rows checked */
  int64_t interior_facets; /* facets shared by two rows */
  int64_t hull_facets;     /* facets of one row only */
  int64_t edges;           /* distinct edges */
  int64_t euler;           /* V - E + T (2D) or V - E + F - T (3D) */
  int64_t bad_index;       /* rows with an index outside [0, n) or a repeated index */
  int64_t flat;            /* rows of zero orientation */
  int64_t non_manifold;    /* facets found in more than two rows */
  int64_t asymmetric;      /* neighbour links that do not match each other */
  int64_t folded;          /* interior facets whose two rows lie on the same side */
  int64_t non_delaunay;    /* interior facets that are not locally Delaunay */
  int64_t non_convex;      /* hull ridges where the boundary bends inwards */
  int64_t unused_points;   /* input points that are a vertex of no row */
  int64_t pivot_limit;     /* hull-ridge walks that hit their step limit (4096) */
  int64_t violations;      /* sum of the eight counters above plus (euler != 1) */
} dt_validation;

/* One entry of the per-kernel profile (profile mode). */
typedef struct dt_kernel_profile {
  char name[32];
  int64_t launches;
  double ms;             /* summed CUDA-event time on the context stream */
  double bytes;          /* algorithmic bytes (each record the kernel must touch, once) */
  double flops;          /* floating-point operations of the first (FP32) predicate stage */
} dt_kernel_profile;

typedef struct dt_ctx dt_ctx;

/* Fill *cfg with the defaults listed in dt_config.  Returns DT_OK. */
DT_API int dt_config_default(dt_config* cfg);

/* Create a context on CUDA device `device`.  `cuda_stream` (a cudaStream_t,
 * may be NULL for a private stream) is the stream every kernel of this
 * context runs on; `cfg` may be NULL for defaults.  *out receives the
 * context (owned by the caller, released by dt_destroy). */
DT_API int dt_create(dt_ctx** out, int device, void* cuda_stream, const dt_config* cfg);

/* Replace the context's configuration (NULL restores the defaults). */
DT_API int dt_set_config(dt_ctx* ctx, const dt_config* cfg);

/* Triangulate n points of dimension dim (2 or 3), points host or device,
 * with k partitions (k >= 1; k = 1 triangulates directly) and sample
 * fraction sample_frac in [0, 1] (0 selects the paper's default
 * eta = ceil(sqrt(n)), Sec. 4.2).  Device points must stay valid until the
 * call returns.  The result replaces the context's previous result.
 * Errors: DT_E_ARG, DT_E_DUPLICATE, DT_E_DEGENERATE, DT_E_NOMEM,
 * DT_E_TIMEOUT, DT_E_OVERFLOW, DT_E_RANGE, DT_E_CUDA, DT_E_INTERNAL. */
DT_API int dt_triangulate(dt_ctx* ctx, const double* points, int64_t n, int dim, int k,
                   double sample_frac);

/* Copy the finite simplices of the last result into out (host or device,
 * room for capacity simplices of dim+1 int32 each).  *count receives the
 * number of simplices; with out == NULL only *count is written.  Returns
 * DT_E_ARG if capacity is too small. */
DT_API int dt_get_simplices(dt_ctx* ctx, int32_t* out, int64_t capacity, int64_t* count);

/* Device pointer to the last result's simplex array (library-owned, valid
 * until the next dt_triangulate or dt_destroy) and its count. */
DT_API int dt_get_simplices_device(dt_ctx* ctx, const int32_t** dptr, int64_t* count);

/* Neighbourhood update of the merge (Alg. 1, the loop after the merge):
 * the neighbours of the last result's simplices, as (dim+1) int32 per
 * simplex in the order of dt_get_simplices.  Entry j of simplex r is the
 * simplex sharing every vertex of r except its j-th, or -1 when that facet
 * lies on the convex hull.  Computed on the first call after dt_triangulate
 * unless dt_config.neighbors made dt_triangulate compute it.  out is host or
 * device with room for capacity simplices; with out == NULL only *count is
 * written.  DT_E_ARG after a batched call (no single result) or when
 * capacity is too small. */
DT_API int dt_get_neighbors(dt_ctx* ctx, int32_t* out, int64_t capacity, int64_t* count);

/* Certify that m simplices (dim+1 int32 vertex indices each, any order
 * within a row, host or device) are the Delaunay triangulation of the n
 * points (row-major float64, host or device) under the same perturbation
 * rule as dt_triangulate; the checks are listed with dt_validation.  The
 * result goes to *out; the call returns DT_OK whether or not the rows pass
 * (bad indices are counted, not errors).  Errors: DT_E_ARG (null pointers,
 * dim, n < dim + 1, m < 0), DT_E_NOMEM, DT_E_RANGE, DT_E_OVERFLOW, DT_E_CUDA.
 * The context's last triangulation result is left untouched. */
DT_API int dt_validate(dt_ctx* ctx, const double* points, int64_t n, int dim, const int32_t* simplices,
                       int64_t m, dt_validation* out);

/* Statistics of the last call. */
DT_API int dt_get_stats(dt_ctx* ctx, dt_stats* stats);

/* Per-point partition label of the last call (host or device out, n int32).
 * All zeros when k = 1 ran. */
DT_API int dt_get_labels(dt_ctx* ctx, int32_t* out, int64_t n);

/* Sample of the last call: eta input indices, ascending (host or device out).
 * *count receives eta; with out == NULL only *count is written. */
DT_API int dt_get_sample(dt_ctx* ctx, int32_t* out, int64_t capacity, int64_t* count);

/* Block of every sample point (eta int32, host or device out). */
DT_API int dt_get_sample_blocks(dt_ctx* ctx, int32_t* out, int64_t capacity);

/* Border vertices of the last call: |vertices(B)| input indices, ascending. */
DT_API int dt_get_border_vertices(dt_ctx* ctx, int32_t* out, int64_t capacity, int64_t* count);

/* Per-kernel profile of the last dt_triangulate (filled only when the
 * configuration has profile = 1): up to max entries into out (host), the
 * number available in *count. */
DT_API int dt_get_kernel_profile(dt_ctx* ctx, dt_kernel_profile* out, int max, int* count);

/* Measured arithmetic roof of the predicate stages: the FMA throughput of
 * the GPU's FP32 (precision 32) or FP64 (precision 64) pipe, in TFLOP/s
 * (2 flops per FMA), the best of `reps` timed launches (1..1000) after one
 * untimed launch of independent FMA chains on every SM.  Needs no context;
 * the caller's current device is unchanged.  Returns DT_OK, DT_E_ARG or
 * DT_E_CUDA. */
DT_API int dt_measure_fma_rate(int device, int precision, int reps, double* tflops);

/* Human-readable description of the last error on this context (never NULL). */
DT_API const char* dt_last_error(dt_ctx* ctx);

/* Release the context and every buffer it owns.  NULL is ignored. */
DT_API void dt_destroy(dt_ctx* ctx);

/* ---- batched form: many independent problems in one call ---- */

/* Triangulate `count` independent point sets of dimension dim in one engine
 * run (one set of kernel launches for all of them).  Instance i is rows
 * offsets[i] .. offsets[i+1]-1 of points (host or device, float64 row-major);
 * offsets: count+1 int64 in HOST memory, offsets[0] = 0, non-decreasing,
 * total below 2^28.  Each instance is triangulated directly (Alg. 1 base
 * case); perturbation ranks are the point order inside each instance.
 * Duplicates are checked inside each instance (DT_E_DUPLICATE); an instance
 * that is flat or has fewer than dim+1 points gets an empty result and a
 * per-instance status (dt_get_batch_status).  Replaces the previous result. */
DT_API int dt_triangulate_batch(dt_ctx* ctx, const double* points, const int64_t* offsets, int count, int dim);

/* Simplices of the last batch: rows of dim+1 int32 INSTANCE-LOCAL vertex
 * indices (each row sorted, rows sorted per instance, instances in order)
 * into out (host or device, capacity rows); out_offsets (host, count+1, may
 * be NULL) receives each instance's first row; *total the row count.  With
 * out == NULL only the counts are written. */
DT_API int dt_get_batch_simplices(dt_ctx* ctx, int32_t* out, int64_t capacity, int64_t* out_offsets,
                                  int64_t* total);

/* Per-instance status of the last batch: 0, DT_E_DEGENERATE (flat) or
 * DT_E_ARG (fewer than dim+1 points); status: count int32 (host). */
DT_API int dt_get_batch_status(dt_ctx* ctx, int32_t* status, int count);

/* ---- asynchronous jobs (systems extension; the paper has no counterpart) ---- */

/* Queue one triangulation, exactly what dt_triangulate(points, n, dim, k,
 * sample_frac) computes, and return at once; *job receives its id (ids start
 * at 1 and are never reused).  The points (host or device, n x dim float64)
 * are copied before the call returns; the caller may free them afterwards.
 * Jobs run in submission order on the context's job worker: a second context
 * on the same device (created by the first dt_submit with this context's
 * configuration) with its own stream, buffers and host thread, so they run
 * alongside this context's own calls.  Argument errors (as dt_triangulate's)
 * are returned here; errors of the triangulation itself by dt_poll.
 * Returns DT_OK, DT_E_ARG, DT_E_CUDA or DT_E_NOMEM. */
DT_API int dt_submit(dt_ctx* ctx, const double* points, int64_t n, int dim, int k, double sample_frac,
                     uint64_t* job);

/* *done = 1 once the job has finished, else 0.  A finished job returns its
 * triangulation's result code (DT_OK or the error, with dt_last_error set);
 * an unknown or released id returns DT_E_ARG. */
DT_API int dt_poll(dt_ctx* ctx, uint64_t job, int* done);

/* A finished job's simplices, in dt_get_simplices' format (rows of dim+1
 * sorted global indices, rows sorted); out: HOST memory, capacity rows, NULL
 * for a size query (*count only).  DT_E_ARG for an unknown or unfinished job;
 * a failed job returns its error code. */
DT_API int dt_get_job_simplices(dt_ctx* ctx, uint64_t job, int32_t* out, int64_t capacity, int64_t* count);

/* Frees a finished job's result; DT_E_ARG for an unknown id or a job still
 * queued or running.  dt_destroy frees every job: it waits for the running
 * one and drops those still queued. */
DT_API int dt_release_job(dt_ctx* ctx, uint64_t job);

/* ---- continuous batching: one resident engine for a stream of jobs ---- */

/* A stream keeps device buffers for `capacity` points (and their simplex
 * arenas) on the context's GPU and triangulates many independent jobs of one
 * dimension in the same insertion rounds.  Between rounds the engine returns
 * to the host, which admits queued jobs into free room (each job an instance
 * with its own insertion schedule) and extracts the jobs whose points are
 * all inserted; a job that arrives while others run starts at the next round
 * boundary.  Each job's result is exactly its DT (the same rows as a
 * dt_triangulate of its points alone).  Not in the paper: a systems form of
 * its per-partition triangulations (Alg. 1) for serving.
 *
 * dt_stream_open: dim 2 or 3; 16 <= capacity < 2^26 points; 1 <= max_jobs <=
 * 1024 jobs resident at once.  One stream per context; it holds about
 * (arena_factor x 48 + 100) bytes per point of capacity plus fixed scratch
 * (dt_stream_get_info reports the total).  DT_E_NOMEM if the device cannot
 * hold it.  The rounds of a stream are numbered over its whole life (the
 * number orders its claims, which are not cleared between jobs), so one
 * stream serves at most 2^31 - 1 insertion rounds, about nine days at the
 * ~2,800 rounds per second of a busy 3D serving load; close and reopen it
 * before that. */
DT_API int dt_stream_open(dt_ctx* ctx, int dim, int64_t capacity, int max_jobs);

/* Queues a job: n points (n x dim float64, HOST memory, copied).  May be
 * called from another host thread than dt_stream_run (the only call with
 * that property).  *job receives its id.  A job needs n + 1 + ceil(32 /
 * arena_factor) points of the capacity while it runs; DT_E_NOMEM if that
 * exceeds the whole stream. */
DT_API int dt_stream_submit(dt_ctx* ctx, const double* points, int64_t n, uint64_t* job);

/* Runs up to `quanta` admission + round-loop passes: each admits queued jobs
 * that fit (in arrival order; a job that does not fit yet lets smaller ones
 * behind it pass), then runs insertion rounds until a job finishes, a new
 * job is queued, or nothing is running; finished jobs are extracted.
 * *pending (optional) receives the running + queued jobs.  A bad job
 * (duplicate or non-finite points: DT_E_DUPLICATE / DT_E_ARG; fewer than
 * dim + 1 or affinely dependent points: DT_E_ARG / DT_E_DEGENERATE) fails
 * alone.  A device error fails every running job with its code and leaves
 * the stream empty and usable; the call then returns that code. */
DT_API int dt_stream_run(dt_ctx* ctx, int quanta, int* pending);

/* Status of a job: 0 queued, 1 running, 2 done (rows in *count, optional),
 * negative: the DT_E_* code it failed with.  DT_E_ARG for an unknown id. */
DT_API int dt_stream_job(dt_ctx* ctx, uint64_t job, int* status, int64_t* count);

/* A done job's simplices in dt_get_simplices' format (rows of dim + 1
 * sorted input indices, rows sorted) into HOST memory; out NULL for a size
 * query.  A failed job returns its code; DT_E_ARG otherwise. */
DT_API int dt_stream_fetch(dt_ctx* ctx, uint64_t job, int32_t* out, int64_t capacity, int64_t* count);

/* Forgets a done or failed job (its rows are freed).  DT_E_ARG for an
 * unknown, queued or running job. */
DT_API int dt_stream_release(dt_ctx* ctx, uint64_t job);

typedef struct dt_stream_info {
  int64_t capacity;      /* points */
  int64_t free_points;   /* points of the capacity not taken by running jobs */
  int64_t device_bytes;  /* device memory the stream holds */
  int32_t running, queued;
  int64_t quanta;        /* round-loop passes so far */
  int64_t rounds;        /* insertion rounds so far */
  int64_t launches;      /* kernels the context has launched so far (every call) */
} dt_stream_info;

DT_API int dt_stream_get_info(dt_ctx* ctx, dt_stream_info* out);

/* Frees the stream (waits for nothing: call it between dt_stream_run calls).
 * dt_destroy closes an open stream too. */
DT_API int dt_stream_close(dt_ctx* ctx);

/* ---- step-level entry points (operate on caller buffers; host or device) ---- */

/* Exact predicate signs for m index tuples into points (n x dim, host or
 * device); gid (n int64, may be NULL for 0..n-1) ranks the perturbation.
 * kind 0: orient of dim+1 points; 1: perturbed insphere of point dim+1
 * against simplex 0..dim (orientation normalised, 0 if flat); 2: raw
 * insphere sign (-1)^dim det[p_i - q, |p_i - q|^2]; 3: sign(|p-a|^2 - |p-b|^2)
 * for tuples (p, a, b).  out: m int8 (host or device).  Runs on the GPU. */
DT_API int dt_eval_predicates(dt_ctx* ctx, const double* points, int64_t n, int dim,
                       const int64_t* gid, int kind, const int32_t* tuples, int64_t m,
                       int8_t* out);

/* Alg. 2 (assignment of the points) on given inputs: label every point of P (n x dim) with
 * block[j] of its exactly nearest sample point S_j (ties: smaller srank),
 * walking the Delaunay graph of S.  All buffers host or device; out n int32. */
DT_API int dt_label_points(dt_ctx* ctx, const double* P, int64_t n, int dim, const double* S,
                    const int64_t* srank, const int32_t* block, int64_t m, int32_t* out);

/* k-way partition of a sample graph given as an edge list (E rows u < v,
 * int64 weights) over eta vertices with coordinates S (eta x dim): the
 * deterministic initial blocks of the context's partition_init (Hilbert runs
 * or the kd median split) refined by label propagation.  out: eta int32. */
DT_API int dt_partition_graph(dt_ctx* ctx, const double* S, int64_t eta, int dim, const int32_t* E,
                       const int64_t* w, int64_t m, int k, double eps, int rounds,
                       int32_t* out);

/* ---- allocation-free variant ---- */

/* Sample selection (the eta smallest keys splitmix64(splitmix64(seed) ^ i),
 * i < n; the same indices dt_triangulate draws for its sample) for callers
 * that cannot allocate device memory: code running inside an allocator or a
 * memory pool it does not own, processes with capped or audited allocations,
 * or real-time paths where cudaMalloc and its implicit synchronisation are
 * not allowed.  The paper has no counterpart; it is a systems entry point.
 *
 * Needs no context and allocates nothing: its scratch is one file-scope
 * device array of 9240 bytes that every GPU loading this library keeps until
 * the process exits.  out_ids: eta int32 in DEVICE memory of `device`
 * (caller-allocated; host pointers and memory of another GPU are rejected
 * with DT_E_ARG before anything runs), written in ascending order.  The
 * caller's current device is the same after the call as before it.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream); the call
 * synchronises it before returning.
 * Limits: 1 <= eta <= n <= 2^31 - 1; anything else returns DT_E_ARG.
 * The first call on a device, with that device current, looks up the
 * array's device address (cudaGetSymbolAddress) and caches it: make that
 * first call before any stream capture.  All calls share the array, which
 * keeps the last call's contents (each call clears what must start at zero);
 * calls that overlap on the GPU race on it and must be ordered by the caller.
 * Returns DT_OK, DT_E_ARG or DT_E_CUDA. */
DT_API int dt_select_sample_noalloc(int device, void* cuda_stream, int64_t n, int64_t eta, uint64_t seed,
                                    int32_t* out_ids);

#ifdef __cplusplus
}
#endif
#endif /* GB300_DT_H */
