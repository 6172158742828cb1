/*
 * mg.h -- C-ABI of the GB300 Mixture Graph library (libmg.so).
 *
 * The Mixture Graph (Al-Thelaya, Agus, Schneider, "The Mixture Graph -- A Data
 * Structure for Compressing, Rendering, and Querying Segmentation Histograms",
 * IEEE Vis 2020) factorises the normalised histogram mipmap of a segmentation
 * volume into binary lerps between segment IDs, so that
 *   - a transfer function on the segments becomes a colour per mipmap voxel by
 *     one forward pass over the lerp DAG (Sec. 3.4, Sec. 4), and
 *   - the segment histogram of a box becomes a footprint of coarse mipmap
 *     samples whose weights are pushed back through the DAG (Sec. 3.6).
 *
 * Conventions for every call:
 *   - Array arguments are device pointers unless a name ends in _host.  The
 *     caller owns them; the library never frees or keeps them.
 *   - Every call is asynchronous on `stream` unless its comment says it
 *     synchronises.  Calls return mg_status and never abort, throw or exit; a
 *     message for the last failure of the calling thread is in mg_last_error().
 *   - Argument errors that the host can see are returned before any launch.
 *     Errors only the device can see (an ID >= num_segments, a malformed box,
 *     an inexact integer push) set the graph's device status word, which
 *     mg_sync_status() reads and clears.
 *   - Volumes are x-fastest: voxel (x, y, z) is element (z*ny + y)*nx + x.
 *     Each axis is at most 65535 voxels and nx*ny*nz < 2^32.
 *   - Node IDs: sources 0..S-1 are the segment IDs; internal nodes S..N-1 are
 *     numbered by ascending (topological level, p, q, a, b), so a node's
 *     predecessors always have smaller IDs (Eq. 8) and nodes of one level are
 *     contiguous (Sec. 3.4).
 */
#ifndef MG_H
#define MG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MG_API __attribute__((visibility("default")))
#else
#define MG_API
#endif

/* cudaStream_t without requiring the CUDA headers */
typedef struct CUstream_st *mg_stream;

#define MG_MAX_LEVELS 32
#define MG_MAX_DEPTH 64
#define MG_NO_NODE 0xFFFFFFFFu

typedef enum {
    MG_OK = 0,
    MG_ERR_INVALID_ARG = 1,  /* bad argument, or bad input data seen on the device */
    MG_ERR_OOM = 2,          /* the allocator returned NULL */
    MG_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    MG_ERR_TIMEOUT = 4,      /* a bounded device-side wait expired */
    MG_ERR_CAPACITY = 5,     /* sparse output larger than the caller's capacity */
    MG_ERR_UNSUPPORTED = 6,  /* size or option outside what this build supports */
    MG_ERR_INEXACT = 7,      /* an integer push met a weight not divisible by a+b */
    MG_ERR_CANCELLED = 8     /* a request of the request loop was cancelled before launch */
} mg_status;

typedef enum { MG_F32 = 0, MG_F16 = 1, MG_BF16 = 2 } mg_dtype;

typedef struct mg_graph mg_graph;   /* opaque, library-owned */

/* Device memory for the graph and for per-call scratch.  alloc returns a
 * device pointer usable in stream order on `stream` (NULL = out of memory),
 * 256-byte aligned as cudaMalloc's (else the call fails with
 * MG_ERR_INVALID_ARG); free releases it in stream order.  Pass NULL to mg_build to use
 * cudaMallocAsync / cudaFreeAsync. */
typedef struct {
    void *ctx;
    void *(*alloc)(void *ctx, size_t bytes, mg_stream stream);
    void (*free)(void *ctx, void *ptr, size_t bytes, mg_stream stream);
} mg_allocator;

typedef struct {
    int id_bytes;      /* 2: ids are uint16, 4: ids are uint32 */
    int reserved[7];   /* zero */
} mg_build_opts;

typedef struct {
    uint32_t num_segments;                    /* S: sources */
    int levels;                               /* L: mip levels, level 0 = input */
    int depth;                                /* D: topological depth */
    int64_t num_nodes;                        /* N: sources + internal nodes */
    int64_t dims[MG_MAX_LEVELS][3];           /* per-level (x, y, z) resolution */
    int64_t bucket[MG_MAX_DEPTH + 2];         /* nodes of level d: [bucket[d], bucket[d+1]) */
    int64_t max_list;                         /* longest mixture of any voxel */
    int64_t pairs;                            /* sum over voxels of (entries - 1) */
    int64_t device_bytes;                     /* bytes the graph holds on the device */
    double build_ms;                          /* wall time of mg_build */
    int64_t lut_entries;                      /* entries of the mixture lookup table (Sec. 3.6) */
} mg_graph_info;

/*
 * mg_build -- build the Mixture Graph of a segmentation volume.
 *   Sec. 3.1 (Eq. 4): normalised histogram mipmap, average-of-eight with N =
 *     children in support at the borders, levels rounding up to 1^3; held as
 *     integer weights 8^l * H.
 *   Sec. 3.2 (Eq. 5-7): each mixture with more than one entry is factorised
 *     into binary lerps.  Pair choice: the entries, sorted by segment ID, are
 *     lerped pairwise (0,1),(2,3),... per round, an odd last entry carried,
 *     until one remains.
 *   Sec. 3.3: identical lerps (same predecessors, same reduced integer ratio
 *     a:b) are one node, so no voxel's mixture changes (exact, no quantiser).
 *   Sec. 3.4 / Fig. 5: topological levels; nodes renumbered canonically.
 * ids: nx*ny*nz segment IDs (uint16 or uint32 per opts->id_bytes), each
 *   < num_segments (else MG_ERR_INVALID_ARG after the build's sync).
 * allocator: may be NULL (cudaMallocAsync).  It is copied into the graph and
 *   used for the graph's memory and for scratch of later calls.
 * Synchronises `stream` several times (level sizes are data dependent).
 * On success *out owns its device memory until mg_free.
 */
MG_API mg_status mg_build(const void *ids, int64_t nx, int64_t ny, int64_t nz,
                          uint32_t num_segments, const mg_build_opts *opts,
                          const mg_allocator *allocator, mg_stream stream, mg_graph **out);

/* Sizes and level geometry of a built graph (host only, no device work). */
MG_API mg_status mg_graph_info_get(const mg_graph *g, mg_graph_info *info);

/* Copy the node table to caller buffers (host or device, any may be NULL):
 * p[N], q[N] predecessors (MG_NO_NODE for sources), a[N], b[N] the coprime
 * weights of p and q (0 for sources).  Node n is the lerp (a*p + b*q)/(a+b),
 * Eq. 5-7.  Synchronises `stream`. */
MG_API mg_status mg_graph_copy_nodes(const mg_graph *g, uint32_t *p, uint32_t *q, uint64_t *a,
                                     uint64_t *b, mg_stream stream);

/* Copy the node ID of every voxel of one level (dims[level], x fastest) to a
 * caller buffer (host or device).  Level 0 gives the segment IDs (lossless,
 * Sec. 3.4).  Synchronises `stream`. */
MG_API mg_status mg_graph_copy_mip(const mg_graph *g, int level, uint32_t *dst, mg_stream stream);

/*
 * mg_propagate_tf -- forward transfer-function propagation (Sec. 3.4, Sec. 4,
 * Sec. 5.2 "Color lookup table").
 *   vals[s] = tf[s] for sources; for every internal node, level by level,
 *   vals[n] = (1 - alpha_n) * vals[p] + alpha_n * vals[q], alpha_n = b/(a+b),
 *   computed in fp32.  The colour of mipmap voxel v at level l is then
 *   vals[node ID of v] (a paletted lookup).
 * tf: S x C fp32, row-major.  C in 1..16.
 * storage: dtype of vals (MG_F32, MG_F16 or MG_BF16).  For 16-bit storage the
 *   node weights are read as 16-bit too (alpha <= 1/2 kept by swapping p and q,
 *   the interpolation symmetry of Sec. 3.7); arithmetic stays fp32.
 * vals: N x C in `storage`, caller-owned, fully overwritten.
 */
MG_API mg_status mg_propagate_tf(mg_graph *g, const float *tf, int C, mg_dtype storage, void *vals,
                                 mg_stream stream);

/*
 * mg_propagate_tf_multi -- k transfer functions propagated in one pass over the
 * graph (Sec. 3.4), e.g. k pending TF updates of one volume: the k*C values of
 * a node are one row, so each level's wait and each predecessor gather serve
 * all k.  Channel c of TF j is channel j*C + c of the row; every channel is
 * the lerp of mg_propagate_tf, so row slice j equals mg_propagate_tf(TF j).
 * tfs: k x S x C fp32 (TF j at tfs + j*S*C, each row-major S x C).
 * k in 1..32, C in 1..16, and k*C one of 1-8, 12, 16, 20, 24, 28, 32
 *   (else MG_ERR_UNSUPPORTED).
 * storage: as for mg_propagate_tf.
 * vals: N x (k*C) in `storage`, caller-owned, fully overwritten; 16-byte
 *   aligned when a row is a multiple of 16 bytes (8-byte when of 8).
 */
MG_API mg_status mg_propagate_tf_multi(mg_graph *g, const float *tfs, int k, int C, mg_dtype storage, void *vals,
                                       mg_stream stream);

/* Query output forms. */
typedef enum { MG_HIST_U32 = 0, MG_HIST_F32 = 1 } mg_hist_type;
typedef enum { MG_LAYOUT_DENSE = 0, MG_LAYOUT_CSR = 1 } mg_layout;
typedef enum { MG_SCHED_BATCHED = 0, MG_SCHED_PLAIN = 1, MG_SCHED_NAIVE = 2 } mg_schedule;

typedef struct {
    int hist_type;      /* MG_HIST_U32: exact integer push; MG_HIST_F32: fp32 push */
    int layout;         /* MG_LAYOUT_DENSE or MG_LAYOUT_CSR */
    int alpha_dtype;    /* fp32 push only: node weights read as MG_F32, MG_F16 or MG_BF16 */
    int schedule;       /* MG_SCHED_BATCHED: persistent work queue over cube chunks;
                           MG_SCHED_PLAIN: one launch per query, one CTA (baseline);
                           MG_SCHED_NAIVE: no footprint assembly, every level-0 voxel
                           of the box counted (brute-force baseline, same results) */
    int chunk_cubes;    /* batched: cubes per work item (0 = tuned default) */
    int block_threads;  /* batched: threads per CTA, 128/256/512 (0 = tuned default) */
    int timing;         /* nonzero: record CUDA events around the plan, main and output
                           stages on `stream` (read them with mg_query_timing) */
    int reserved;       /* zero */
} mg_query_opts;

/*
 * mg_query_boxes -- segment histograms of axis-aligned boxes (Sec. 3.6).
 *   Each box (x, y, z, dx, dy, dz) covers [x, x+dx) x [y, y+dy) x [z, z+dz),
 *   clipped to the volume.  It needs 0 <= x < nx (likewise y, z) and dx, dy,
 *   dz >= 1; a box that breaks this sets MG_ERR_INVALID_ARG in the status word
 *   and its histogram is left zero.
 *   Footprint assembly (Algorithm 1): each axis range splits into aligned
 *   power-of-two runs; every block of their tensor product is tiled by cubes
 *   of its shortest side 2^l, one level-l voxel each, weight 8^l.  The weight
 *   is pushed from the voxel's node to the sources in descending topological
 *   order: p receives W*a/(a+b), q receives W*b/(a+b).  Every cube lies inside
 *   the box, so with MG_HIST_U32 the histogram equals the count of level-0 IDs
 *   in the clipped box exactly.
 * boxes: Q x 6 int32.  Q >= 0 (Q = 0 writes only offsets[0] = 0 in CSR).
 * Dense layout: out is Q x S (uint32 or fp32), fully overwritten; seg and
 *   offsets are unused; out_capacity >= Q*S elements.
 * CSR layout: offsets[Q+1] (uint64), seg[nnz] (uint32) and out[nnz] hold each
 *   query's non-zero segments in ascending order.  If nnz > out_capacity the
 *   call returns MG_ERR_CAPACITY with *out_required = nnz and offsets written.
 *   CSR synchronises `stream` once to read nnz.
 * Scratch is allocated from the graph's allocator and released in stream
 * order before return.
 */
MG_API mg_status mg_query_boxes(const mg_graph *g, const int32_t *boxes, int64_t Q,
                                const mg_query_opts *opts, void *out, size_t out_capacity,
                                uint32_t *seg, uint64_t *offsets, size_t *out_required,
                                mg_stream stream);

/*
 * mg_query_boxes_noalloc -- the exact box histograms of mg_query_boxes
 * (uint32 counts, dense Q x S layout, batched schedule, default tuning) for
 * callers that must not allocate device memory: real-time frame loops that
 * cannot absorb an allocation's latency or failure in the middle of a frame,
 * engines whose memory manager reserves the whole device up front and lets no
 * library allocate, and services held to a fixed memory budget.  The paper has
 * no counterpart; this is a deployment aid.
 * Its scratch is a 64 MiB array compiled into the library (every GPU that
 * loads libmg holds it until the process exits), so the call allocates
 * nothing.  A batch must fit it: up to about 500,000 boxes, and footprint
 * blocks and chunks of at most 32 MiB (12 bytes per block, 8 per chunk);
 * larger batches return MG_ERR_CAPACITY with `out` left unchanged and the
 * limit in mg_last_error() -- split them.
 * The first call on a device looks up the array's device address (so make
 * it before any stream capture).  All calls share the one array and leave
 * their scratch in it: calls that overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller.
 * out: Q x S uint32, fully overwritten.  Synchronises `stream` once (the
 * footprint size depends on the boxes).  Errors as for mg_query_boxes.
 */
MG_API mg_status mg_query_boxes_noalloc(const mg_graph *g, const int32_t *boxes, int64_t Q, uint32_t *out,
                                        size_t out_capacity, mg_stream stream);

/* Stage durations of the last mg_query_boxes call on this graph made with
 * opts->timing set: plan (footprint plan and scans), main (the histogram
 * kernel or, for MG_SCHED_PLAIN, all per-box launches) and output (dense fp32
 * or CSR finalisation), in milliseconds from CUDA events on that call's
 * stream.  Waits for the call's last event.  Returns MG_ERR_INVALID_ARG if no
 * timed call was made. */
MG_API mg_status mg_query_timing(const mg_graph *g, float *plan_ms, float *main_ms, float *output_ms);

/*
 * Query plans: the batched pipeline of mg_query_boxes for up to max_Q boxes,
 * captured once as a CUDA graph with every buffer preallocated, so that a run
 * is one small kernel (the batch size and the caller's buffers) and one graph
 * launch, with no copies and no host synchronisation.
 * opts: dense layout and batched schedule only; hist_type, alpha_dtype and the
 *   launch shape (0 = the graph's tuned shape, else the defaults) as for
 *   mg_query_boxes.
 * max_blocks, max_chunks: footprint blocks and work chunks one run may need
 *   (0 = 1024 and 256 per box).  A run whose boxes need more writes zero
 *   histograms and sets MG_ERR_CAPACITY in the status word (mg_sync_status).
 * opts->timing set: the graph also records CUDA events around its plan stage
 *   (tile reset and the fused plan kernel) and its main kernel; read the
 *   durations of the last run with mg_query_plan_timing.
 * The plan holds its memory (from the graph's allocator) until
 * mg_query_plan_free; runs of one plan share it, so runs of one plan on
 * different streams must not overlap.
 */
typedef struct mg_query_plan mg_query_plan;
MG_API mg_status mg_query_plan_create(mg_graph *g, int64_t max_Q, const mg_query_opts *opts, int64_t max_blocks,
                                      int64_t max_chunks, mg_query_plan **out);
/* boxes: Q x 6 int32 (device), 0 <= Q <= max_Q; out: Q x S (uint32 or fp32),
 * both 4-byte aligned.  The graph reads `boxes` and writes `out` in the order
 * of `stream`: they must stay valid until the run has completed on it. */
MG_API mg_status mg_query_plan_run(mg_query_plan *p, const int32_t *boxes, int64_t Q, void *out, size_t out_capacity,
                                   mg_stream stream);
/* Durations in milliseconds of the last run's plan stage and main kernel, for a
 * plan created with opts->timing; waits for that run's main kernel.
 * MG_ERR_INVALID_ARG: NULL argument, a plan made without timing, or no run yet. */
MG_API mg_status mg_query_plan_timing(const mg_query_plan *p, float *plan_ms, float *main_ms);
MG_API void mg_query_plan_free(mg_query_plan *p);

/* Autotuner of the batched query: times every work-chunk size in
 * {1024, 2048, 4096, 8192, 16384} cubes with CTAs of 128, 256 and 512 threads on the
 * given batch (dense layout; opts->hist_type and alpha_dtype as the caller
 * will use them), writes the fastest into opts->chunk_cubes/block_threads and
 * keeps it in the graph for later calls and plans that leave them 0.
 * *best_ms (may be NULL) receives the fastest time of one call.
 * Synchronises `stream`. */
MG_API mg_status mg_query_autotune(mg_graph *g, const int32_t *boxes, int64_t Q, mg_query_opts *opts,
                                   float *best_ms, mg_stream stream);
/* Record a tuned launch shape for a histogram type (e.g. from a cache file). */
MG_API mg_status mg_query_set_tuning(mg_graph *g, int hist_type, int chunk_cubes, int block_threads);

/* Number of footprint-assembly cubes (mipmap fetches) of each box, uint64[Q]
 * (the "fetches" of Table 3).  Boxes as for mg_query_boxes. */
MG_API mg_status mg_count_cubes(const mg_graph *g, const int32_t *boxes, int64_t Q, uint64_t *cubes,
                                mg_stream stream);

/*
 * mg_render_lookup -- ray-sample node lookup (Sec. 4: rendering from the graph
 * is a paletted lookup).  Sample i = (x, y, z, lod) in level-0 voxel units.
 *   level = floor(lod + 1/2) in fp32, clamped to [0, L-1] (NaN: 0);
 *   voxel = floor of each coordinate clamped to [0, dim] (NaN: 0), shifted
 *           right by level and clamped to the level's last voxel;
 *   out[i] = vals[node ID of that voxel] (C values of dtype, copied exactly).
 * samples: P x 4 fp32.  vals: N x C in dtype (from mg_propagate_tf).
 * out: P x C in dtype.
 */
MG_API mg_status mg_render_lookup(const mg_graph *g, const void *vals, int C, mg_dtype dtype,
                                  const float *samples, int64_t P, void *out, mg_stream stream);

/*
 * mg_render_lookup_multi -- ray-sample lookups of k frames in one launch, each
 * frame against its own slice of a k-TF palette (vals from
 * mg_propagate_tf_multi): samples [offsets[j], offsets[j+1]) belong to frame
 * j, and sample i of frame j gets channels [j*C, (j+1)*C) of the row of the
 * node under it, chosen exactly as by mg_render_lookup (Sec. 4).
 * offsets: k + 1 int64 in HOST memory, offsets[0] = 0, non-decreasing.
 * samples: offsets[k] x 4 fp32.  vals: N x (k*C) in dtype.
 * out: offsets[k] x C in dtype.
 */
MG_API mg_status mg_render_lookup_multi(const mg_graph *g, const void *vals, int k, int C, mg_dtype dtype,
                                        const float *samples, const int64_t *offsets, void *out, mg_stream stream);

/*
 * mg_raymarch -- direct volume rendering from the graph (Sec. 4) into a
 * headless image.  For pixel (i, j) (row 0 at the top) the ray leaves `eye`
 * along fwd + ((i + 1/2 - W/2) pix) right + ((H/2 - j - 1/2) pix) up,
 * normalised, and is clipped to the volume [0, nx] x [0, ny] x [0, nz]
 * (level-0 voxel units, voxel v covering [v, v+1)).  Samples lie on the
 * lattice t_k = t_start + k * base_step.  A sample's LOD is floor(log2(t *
 * pix)) + lod_bias (pixel coverage linear in depth); it picks level m = the
 * LOD clamped to [0, L-1] and the step 2^m * base_step (the next sample is
 * k + 2^m).  The sample's value is trilinear within level m between the 8
 * voxel centres around it (clamped to the level) and, when the LOD lies
 * between m and m+1 < L, linear between the two levels by the fractional LOD
 * (quadrilinear).  Opacity correction for the step: alpha' = 1 - (1 -
 * alpha)^(2^m).  Compositing is front to back with weight (1 - A) alpha' on
 * the sample's colour; the ray stops once A >= ert (ert > 1: never) or after
 * max_steps lattice steps.
 * Empty-space skipping (opacity not NULL): opacity[n] is node n's opacity
 * (the TF's alpha propagated through the graph, e.g. mg_propagate_tf with
 * C = 1); climbing from level m+2 while the voxel around the sample has
 * opacity exactly 0, the lattice samples inside the largest such voxel
 * shrunk by 3 * 2^m on every side (the reach of the interpolation), and
 * before the LOD changes, are skipped.  Each would add exactly nothing, so
 * the image equals the one without skipping.  The climbs read a bit mask
 * of the voxels of levels >= 2 whose opacity is non-zero, built first in the
 * graph's per-stream scratch (one pass over those levels' IDs).
 * Decisions (lattice, level, skips, termination) are taken in fp32 with one
 * rounding per operation.
 * vals: N x 4 fp32 node values (mg_propagate_tf, storage MG_F32), 16-byte
 *   aligned.  cam: host struct.  image: H x W x 4 fp32 (R, G, B, A), 16-byte
 *   aligned.  steps (may be NULL): H x W int32 samples composited per pixel.
 */
typedef struct {
    float eye[3], fwd[3], right[3], up[3];   /* level-0 voxel units; fwd, right, up orthonormal */
    float pix;                               /* angle of one pixel (radians) */
    int32_t width, height;                   /* image size, 1..16384 each */
    float base_step;                         /* lattice step in level-0 voxels, > 0 */
    int32_t lod_bias;                        /* added to floor(log2(t * pix)) */
    float ert;                               /* early-termination opacity; > 1: none */
    int32_t max_steps;                       /* lattice steps at most, >= 1 */
    int32_t reserved[4];                     /* zero */
} mg_camera;

MG_API mg_status mg_raymarch(const mg_graph *g, const float *vals, const float *opacity, const mg_camera *cam,
                             float *image, int32_t *steps, mg_stream stream);

/*
 * Request loop (serving).  A server keeps the graphs of several volumes
 * resident on one GPU and runs box-histogram requests (Sec. 3.6) and
 * TF-update frames (propagation, Sec. 3.4, then ray-sample lookups, Sec. 4)
 * as they arrive.  A worker thread owns `slots` CUDA streams.  Whenever a
 * slot is free it takes the oldest queued request; a box request takes with
 * it the next queued boxes of the same volume, in arrival order, while they
 * fit the slot's batch (max_batch boxes and the footprint capacity of the
 * slot's captured query plan), and the whole batch runs as one plan launch;
 * a TF frame takes with it
 * the next queued frames of its volume (up to 8, as long as frames * C is a
 * channel count of mg_propagate_tf_multi), propagated in one pass and looked
 * up in one launch.
 * Requests that arrive while slots are busy join the next batch, so batches
 * of different volumes overlap on the device (continuous batching).  The
 * paper evaluates single queries; the loop is a deployment layer around its
 * operations.
 *
 * Memory: every admitted volume gets, per slot, a query plan and staging
 * buffers (device and pinned host) sized by the options.  A volume whose
 * graph plus these buffers would take the server past memory_budget is not
 * admitted (MG_ERR_CAPACITY), so resident volumes never compete for memory
 * at run time.
 */
typedef struct mg_server mg_server;   /* opaque */

typedef struct {
    int slots;              /* concurrent streams (0 = 4; at most 64) */
    int max_batch;          /* boxes per launch (0 = 1024; at most 2^20) */
    int hist_type;          /* MG_HIST_U32 (exact counts) or MG_HIST_F32 */
    int storage;            /* TF frames: node values as MG_F32, MG_F16 or MG_BF16 */
    int64_t max_samples;    /* TF frames: ray samples per frame (0 = 65536) */
    int64_t memory_budget;  /* bytes the admitted volumes may hold (0 = no limit) */
    int plain;              /* 1: no batching, every box is its own one-CTA launch
                               (the one-launch-per-query baseline under the same traffic) */
    int reserved[5];        /* zero */
} mg_server_opts;

typedef enum { MG_REQ_BOX = 0, MG_REQ_TF = 1 } mg_request_kind;

typedef struct {
    int kind;               /* mg_request_kind */
    int volume;             /* index returned by mg_server_add_volume */
    int32_t box[6];         /* MG_REQ_BOX: (x, y, z, dx, dy, dz) as for mg_query_boxes */
    const float *tf;        /* MG_REQ_TF: S x C fp32 transfer function (host) */
    const float *samples;   /* MG_REQ_TF: P x 4 fp32 samples as for mg_render_lookup (host) */
    int64_t P;              /* MG_REQ_TF: number of samples, 0..max_samples */
    void *result;           /* host, may be NULL.  MG_REQ_BOX: S counts (uint32, or fp32 with
                               MG_HIST_F32).  MG_REQ_TF: P x C values in the storage dtype */
    double arrival_s;       /* mg_server_replay only: arrival time in seconds from its start */
} mg_request;

typedef struct {
    int64_t box_requests;   /* completed box requests */
    int64_t tf_requests;    /* completed TF frames */
    int64_t box_launches;   /* box batches launched (plan runs, or plain launches) */
    int64_t max_batch_seen; /* largest box batch */
    int64_t cancelled;      /* requests cancelled before launch */
    int64_t failed;         /* requests that completed with an error */
    int64_t memory_admitted; /* bytes the admitted volumes hold (graphs, plans, buffers) */
    int64_t tf_launches;    /* TF work items launched (each up to 8 frames of one volume) */
} mg_server_stats;

/* Create a server on the current device.  opts may be NULL (defaults).
 * Invalid options: MG_ERR_INVALID_ARG before any CUDA call. */
MG_API mg_status mg_server_create(const mg_server_opts *opts, mg_server **out);

/* Admit a volume: its graph g (built with mg_build, owned by the caller and
 * kept alive until it is removed or the server freed) and the channel count C
 * (1-8, 12 or 16) of its TF frames -- before or while serving (from one
 * thread at a time).  Allocates the volume's per-slot plans and buffers from
 * g's allocator, runs each slot's scratch up to size (serving then allocates
 * nothing for it) and synchronises the device.  MG_ERR_CAPACITY if the
 * budget's remainder does not hold it (nothing is kept) or 1024 volumes were
 * admitted.  *volume = its index (indices are never reused). */
MG_API mg_status mg_server_add_volume(mg_server *sv, mg_graph *g, int C, int *volume);

/* Remove (evict) a volume: new requests for it fail; before the start its
 * queued requests are cancelled, after it the call waits (up to timeout_s, 0
 * = no limit: else MG_ERR_TIMEOUT and the volume stays) until no queued or
 * running work refers to it; then its per-slot plans and buffers are freed
 * and their bytes return to the budget.  The graph stays the caller's; it
 * can be admitted again (under a new index). */
MG_API mg_status mg_server_remove_volume(mg_server *sv, int volume, double timeout_s);

/* Start the worker thread. */
MG_API mg_status mg_server_start(mg_server *sv);

/* Queue a request (thread-safe; before mg_server_start requests wait in the
 * queue).  The request is copied; tf, samples and result must stay valid
 * until it completes.  Checked on the host: volume,
 * kind, box bounds (MG_ERR_INVALID_ARG), P <= max_samples, and a box whose
 * footprint alone exceeds a slot's plan capacity (MG_ERR_CAPACITY).
 * *ticket identifies it for mg_server_wait / mg_server_cancel. */
MG_API mg_status mg_server_submit(mg_server *sv, const mg_request *r, uint64_t *ticket);

/* Cancel a queued request: MG_OK if it had not been launched (its wait then
 * returns MG_ERR_CANCELLED), MG_ERR_INVALID_ARG if it was already launched,
 * done or unknown. */
MG_API mg_status mg_server_cancel(mg_server *sv, uint64_t ticket);

/* Wait for a request (thread-safe).  *latency_s (may be NULL) = seconds from
 * its submission (or replay arrival) to its result being in host memory.
 * Returns the request's status; MG_ERR_TIMEOUT if it is not done within
 * timeout_s seconds (0 = no limit), leaving it queued or running. */
MG_API mg_status mg_server_wait(mg_server *sv, uint64_t ticket, double timeout_s, double *latency_s);

/* Replay a timed request stream: submits reqs[i] at reqs[i].arrival_s
 * (non-decreasing, seconds from the start of the call) from the calling
 * thread, then waits for all of them.  latency_s[i] (may be NULL) is measured
 * from the scheduled arrival, so queueing behind a late submission counts.
 * *wall_s (may be NULL) = seconds from the start to the last completion.
 * Returns the first failing request's status (the rest still complete). */
MG_API mg_status mg_server_replay(mg_server *sv, const mg_request *reqs, int64_t n, double *latency_s,
                                  double *wall_s);

/* Counters since creation. */
MG_API mg_status mg_server_stats_get(mg_server *sv, mg_server_stats *stats);

/* Stop the worker (queued requests complete with MG_ERR_CANCELLED), wait for
 * launched work and release the server's memory.  The graphs stay the
 * caller's.  NULL is ignored. */
MG_API void mg_server_free(mg_server *sv);

/* Synchronise `stream`, read and clear the graph's device status word.
 * Returns MG_OK or the first error recorded by an earlier call's kernels. */
MG_API mg_status mg_sync_status(mg_graph *g, mg_stream stream);

/*
 * Checkpoint / resume: a built graph as one image in host memory (a header
 * with the sizes, geometry and depth buckets, then the raw device arrays:
 * mip levels and their axis copies, node table, weights, mixture lookup
 * table).  The paper stores its graph as a bit-packed stream (Table 1); this
 * image trades size for a load without any rebuild.
 * mg_graph_export_size: bytes the image needs.
 * mg_graph_export: writes the image into `host` (at least that many bytes);
 *   synchronises `stream`.  MG_ERR_CAPACITY if `bytes` is too small.
 * mg_graph_import: a new graph (device memory from `allocator`, NULL =
 *   cudaMallocAsync) on the current device from an image; the header and every
 *   array size are checked first (MG_ERR_INVALID_ARG for a corrupt or short
 *   image, MG_ERR_UNSUPPORTED for another version).  Synchronises `stream`;
 *   the image may be freed on return.  16-bit weights are rebuilt on demand.
 */
MG_API mg_status mg_graph_export_size(const mg_graph *g, size_t *bytes);
MG_API mg_status mg_graph_export(const mg_graph *g, void *host, size_t bytes, mg_stream stream);
MG_API mg_status mg_graph_import(const void *host, size_t bytes, const mg_allocator *allocator, mg_stream stream,
                                 mg_graph **out);

/*
 * Bitstream (Sec. 3.3, Table 1, Eq. 14-15): the graph as the paper's fixed-
 * rate stream.  Bit i of the stream is bit i % 8 of byte i / 8 and every
 * field is written least significant bit first, in Table 1's order:
 *   (1) sources, 32 bits;  (2) fractional input, 1 bit (0);  (3) bits per node
 *   ID nb = ceil(log2 N), stored minus one in 6 bits;  (4) sigma_max, 32 bits
 *   (0: no quantiser);  (5) resolution, 3 x 32 bits;  (6) quantisation
 *   bitrate minus one, 4 bits (0);  (7) internal nodes N - S, nb bits;
 *   lossless extension (Table 1 has no exact form): 1 bit "exact weights" (1)
 *   and the weight width w minus one in 6 bits;
 *   per level l = 0..L-1: (8) voxel bits r(l) = ceil(log2(i_max(l) - i_min(l)
 *   + 1)) and (9) i_min(l), nb bits each;
 *   (A) every level's voxels x fastest: node ID - i_min(l) at r(l) bits;
 *   (B) every internal node S..N-1: p and q at nb bits, the coprime weights a
 *   and b at w bits (in place of a codebook index);  (C) empty;
 *   zero padding to a multiple of 8 bytes.
 * mg_bitstream_size: the stream's bytes (synchronises: the per-level ID
 *   ranges are reduced on the device).
 * mg_bitstream_write: the stream into `dst` (device, 8-byte aligned, at
 *   least that many bytes); synchronises `stream`.
 * mg_bitstream_parse: the layout from the stream's first bytes (host; the
 *   header is at most ~600 bytes): MG_ERR_INVALID_ARG for a short or
 *   inconsistent header, MG_ERR_UNSUPPORTED for a fractional or quantised one.
 * mg_bitstream_decode_mip / _nodes: a level's node IDs (dims[level], x
 *   fastest) / the node table (as mg_graph_copy_nodes, any pointer may be
 *   NULL), decoded on the device from the stream (device) into device buffers.
 * mg_bitstream_lookup: mg_render_lookup with every sample's node ID read by
 *   bit address from the stream (Sec. 4: voxel data addressed by bit), vals
 *   from a propagation of the same graph.
 */
typedef struct {
    uint32_t num_segments;                   /* S */
    int levels;                              /* L */
    int node_bits;                           /* nb */
    int weight_bits;                         /* w */
    int64_t num_nodes;                       /* N */
    int64_t dims[MG_MAX_LEVELS][3];
    int32_t voxel_bits[MG_MAX_LEVELS];       /* r(l) */
    int64_t imin[MG_MAX_LEVELS];             /* i_min(l) */
    int64_t level_bit[MG_MAX_LEVELS];        /* bit offset of each level's section (A) */
    int64_t node_bit;                        /* bit offset of section (B) */
    int64_t header_bits;                     /* bits before section (A) */
    int64_t bytes;                           /* stream size */
} mg_bitstream_info;

MG_API mg_status mg_bitstream_size(const mg_graph *g, size_t *bytes);
MG_API mg_status mg_bitstream_write(const mg_graph *g, void *dst, size_t bytes, mg_stream stream);
MG_API mg_status mg_bitstream_parse(const void *host, size_t bytes, mg_bitstream_info *info);
MG_API mg_status mg_bitstream_decode_mip(const void *stream_dev, const mg_bitstream_info *info, int level,
                                         uint32_t *out, mg_stream stream);
MG_API mg_status mg_bitstream_decode_nodes(const void *stream_dev, const mg_bitstream_info *info, uint32_t *p,
                                           uint32_t *q, uint64_t *a, uint64_t *b, mg_stream stream);
MG_API mg_status mg_bitstream_lookup(const void *stream_dev, const mg_bitstream_info *info, const void *vals, int C,
                                     mg_dtype dtype, const float *samples, int64_t P, void *out, mg_stream stream);

/*
 * Greedy factorisation (Sec. 3.3, Eq. 10-13; Sec. 3.7): the paper's encoder,
 * on the GPU.  H is every mixture of levels 1..L-1 (Eq. 4, integer weights
 * 8^l H).  Stage 1 repeats rounds: every pair i < j of components that occur
 * together in a mixture with more than tau components is scored -- phi_1
 * (max-occurrence) adds 1 per mixture, phi_2 (max-reduction) adds |h| - 1
 * if |h| > 2, else 2 -- the highest score wins (ties to the smallest (i,
 * j)) and every such mixture holding both has i and j replaced by their
 * lerp with the summed weight.  Stage 2 runs in waves: every mixture left
 * with two or more components lerps its two lowest-numbered ones.  A lerp of
 * p < q with weights c_p, c_q is the node (p, q, a, b) of the reduced ratio
 * a:b = c_p:c_q (bitrate 0: exact), or (p, q, k, 0) with k = floor(c_q 2^b /
 * (c_p + c_q)) (a b-bit scalar quantiser of equal bins over (0, 1); the
 * codeword of bin k is its centre (2k + 1) / 2^(b+1), its sigma the rms of
 * the weights' distance to it; lerps of one pair in one bin are one node).
 * New nodes are numbered in creation order, a round's or wave's in the scan
 * order of the first mixture making them; the result is renumbered as
 * mg_build's graph (level, p, q, a, b).
 * ids: device, as for mg_build (opts->id_bytes; NULL: uint16).  Synchronises
 * `stream` once per round and wave; device memory from cudaMallocAsync.  The
 * result lives in host memory until mg_greedy_free.
 * MG_ERR_UNSUPPORTED when the pair table would exceed 2^30 entries.
 */
typedef struct mg_greedy mg_greedy;   /* opaque */
typedef struct {
    int strategy;      /* 1: phi_1 max-occurrence; 2: phi_2 max-reduction */
    int tau;           /* stage-1 cutoff, >= 1 (the paper uses 3) */
    int bitrate;       /* 0: exact ratios; 1..16: quantiser bits */
    int reserved[5];   /* zero */
} mg_greedy_opts;
typedef struct {
    uint32_t num_segments;
    int levels;
    int depth;
    int reserved0;
    int64_t num_nodes;     /* N, sources included */
    int64_t picks;         /* stage-1 rounds */
    int64_t waves;         /* stage-2 waves */
    double ms;             /* wall time of mg_factor_greedy */
} mg_greedy_info;

MG_API mg_status mg_factor_greedy(const void *ids, int64_t nx, int64_t ny, int64_t nz, uint32_t num_segments,
                                  const mg_build_opts *opts, const mg_greedy_opts *gopts, mg_stream stream,
                                  mg_greedy **out);
MG_API mg_status mg_greedy_info_get(const mg_greedy *r, mg_greedy_info *info);
/* host buffers of N entries (any may be NULL): p, q predecessors (MG_NO_NODE
 * for sources); a, b the exact coprime weights, or for a quantised graph the
 * bin in a and 0 in b */
MG_API mg_status mg_greedy_copy_nodes(const mg_greedy *r, uint32_t *p, uint32_t *q, uint64_t *a, uint64_t *b);
/* host buffer of dims[level] node IDs, x fastest */
MG_API mg_status mg_greedy_copy_mip(const mg_greedy *r, int level, uint32_t *dst);
/* host buffer of 2 * picks uint32: the stage-1 picks (i, j) in creation numbering */
MG_API mg_status mg_greedy_copy_picks(const mg_greedy *r, uint32_t *picks);
/* host buffers of 2^bitrate doubles (quantised graphs) */
MG_API mg_status mg_greedy_copy_codebook(const mg_greedy *r, double *codebook, double *sigma);
MG_API void mg_greedy_free(mg_greedy *r);

/* A graph from a quantised greedy result (bitrate >= 1), on the current
 * device (memory from `allocator`, NULL = cudaMallocAsync): node weights are
 * the codewords of their bins, so propagation, lookups, ray marching, fp32
 * box queries and the mixture table below work on it as on mg_build's
 * graphs; exact-count queries (MG_HIST_U32) return MG_ERR_UNSUPPORTED, as
 * do the bitstream and the export.  Synchronises `stream`.  The result may be
 * freed afterwards. */
MG_API mg_status mg_graph_from_greedy(const mg_greedy *r, const mg_allocator *allocator, mg_stream stream,
                                      mg_graph **out);

/*
 * The mixture lookup table with uncertainties (Sec. 3.5, Eq. 16-17; Sec. 3.6).
 * Row n lists the sources under node n (ascending) with mu, their share of
 * n's mixture, and dmu, its uncertainty: for n the lerp of p and q with
 * weight w of q and uncertainty dw,
 *   mu_i(n) = (1 - w) mu_i(p) + w mu_i(q),
 *   dmu_i(n)^2 = mu_i(n)^2 ((dmu_i(p)/mu_i(p))^2 + (dmu_i(q)/mu_i(q))^2
 *                + 2 (dw/w)^2)   (Eq. 17),
 * a ratio term being 0 for a component absent from that input; sources have
 * mu = 1, dmu = 0.  w = b/(a+b) and dw = 0 for exact graphs; the bin's
 * codeword and sigma for quantised ones.  fp64.
 * mg_error_table_build: builds the table once (synchronises); *entries (may
 *   be NULL) = its entries.  MG_ERR_UNSUPPORTED above 2^31 entries.
 * mg_error_table_copy: the table into host or device buffers (any NULL):
 *   off[N+1] (int64), src/mu/dmu[entries]; unused slack entries (none for
 *   graphs whose lerps join disjoint sources) hold source 2^32 - 1.
 * mg_query_lut: box histograms summed from the table (the paper's query,
 *   Sec. 3.6): hist[q][s] = sum over the box's footprint cubes c (Algorithm
 *   1) of 8^l mu_s(node_c); err[q][s] = sqrt(sum_c (8^l dmu_s(node_c))^2)
 *   (Eq. 16), the error bar.  Boxes as for mg_query_boxes; hist and err
 *   (may be NULL) Q x S fp64, device.  One CTA per box; S <= 12800.
 */
MG_API mg_status mg_error_table_build(mg_graph *g, int64_t *entries, mg_stream stream);
MG_API mg_status mg_error_table_copy(const mg_graph *g, int64_t *off, uint32_t *src, double *mu, double *dmu);
MG_API mg_status mg_query_lut(const mg_graph *g, const int32_t *boxes, int64_t Q, double *hist, double *err,
                              mg_stream stream);

/* Self-test of failure handling: one GPU thread waits, with the same bounded
 * wait the single-pass propagation uses between topological levels (Sec. 3.4),
 * on a device flag that is already set (satisfied = 1: returns MG_OK) or that
 * nothing ever sets (satisfied = 0: after spin_limit polls of >= 100 ns the
 * wait gives up and the call returns MG_ERR_TIMEOUT).  The GPU is neither
 * faulted nor hung and stays usable.  spin_limit: 1..2^22 (the propagation
 * uses 2^22).  Synchronises `stream`.  The paper has no counterpart. */
MG_API mg_status mg_selftest_bounded_wait(int satisfied, unsigned spin_limit, mg_stream stream);

/* Release the graph's device memory (stream-ordered on the build stream's
 * allocator semantics; synchronises the device first).  NULL is ignored. */
MG_API void mg_free(mg_graph *g);

/* Message of the calling thread's last failed call ("" if none). */
MG_API const char *mg_last_error(void);

/* Library version string. */
MG_API const char *mg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MG_H */
