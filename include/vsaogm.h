/*
 * vsaogm.h - C ABI of libvsaogm.so, the GB300 (sm_103a) hot path of VSA-OGM
 * (Snyder et al., "Brain Inspired Probabilistic Occupancy Grid Mapping with
 * Vector Symbolic Architectures", arXiv 2408.09066).
 *
 * The library encodes labelled 2D points as FHRR hypervectors and bundles them
 * into per-tile, per-class memories (Sec. III-B4), decodes the memories over
 * the grid cells (Sec. III-B5) and turns the class maps into occupancy
 * probabilities with the disk-mask entropy filter, softmax and probabilistic
 * signed difference (Algorithm 2, Eqs. softmax, psd, classification).
 *
 * Conventions used by every call
 *  - Pointers named *_dev are CUDA device pointers (or managed memory); *_host
 *    are host pointers (pinned memory is fastest).  The caller owns every
 *    buffer it passes; the library owns the map, its memories, its frequency
 *    tables and its scratch.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Calls only enqueue work on that stream and return; results are
 *    valid once the stream has reached them.  Consecutive calls on one map
 *    must use one stream, or the caller must order them.  A map is not
 *    thread-safe; distinct maps are independent.
 *  - Return value: VSAOGM_OK (0) or a negative VSAOGM_E_* code.  Nothing else
 *    crosses the ABI; vsaogm_last_error() describes the last failure of the
 *    calling thread.  A failed call enqueues nothing.
 *  - Layouts are row-major with x fastest.  A class map is float [H][W]
 *    (row j = y index, column i = x index); two class maps are [2][H][W] with
 *    class 0 = empty (psi = 0) first and class 1 = occupied (psi = 1) second.
 *    Points are float32 pairs (x, y) in metres, [n][2]; labels are uint8 [n].
 *  - Memories are complex64 (interleaved re, im) [2T][D], memory 2*beta + psi
 *    for tile beta = by * tiles_x + bx (Algorithm 1).  They are kept in the
 *    tile-centred frame: memory 2*beta + psi equals the paper's memory times
 *    the unit phasor exp(-i 2 pi nu . mu_beta), mu_beta the tile centre, which
 *    cancels exactly in the similarity of Eq. loc-query.
 */
#ifndef VSAOGM_H
#define VSAOGM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define VSAOGM_OK 0
#define VSAOGM_E_INVAL -1   /* bad argument or configuration            */
#define VSAOGM_E_NOMEM -2   /* a device or host allocation failed         */
#define VSAOGM_E_CUDA -3    /* a CUDA call failed (message has details)   */
#define VSAOGM_E_TIMEOUT -4 /* a bounded device-side wait gave up         */
#define VSAOGM_E_DATA -5    /* input data rejected (checked mode only)    */

/* Arithmetic of the decode contraction (Eq. loc-query). */
#define VSAOGM_DECODE_FP32 0   /* FP32 SIMT, the reference GPU path          */
#define VSAOGM_DECODE_BF16X3 1 /* tensor cores, split hi/lo bf16, FP32 accum */
#define VSAOGM_DECODE_FP16X3 2 /* tensor cores, split hi/lo fp16, FP32 accum */
#define VSAOGM_DECODE_FP8X3 3  /* tensor cores, split hi/lo e4m3, FP32 accum:
                                  about 7 significant bits per product, the
                                  precision study's lowest rung and the
                                  lower-accuracy path: P is off by about 2^-8
                                  in absolute terms, which meets the stated
                                  occupancy bound on lidar-shaped maps but not
                                  on maps whose maximum P is near 1 (few,
                                  spread-out points)                         */

/* vsaogm_config.decode_mode: the toggles of the decoding ablation
 * (Sec. IV-D1: P_hat = f_ACT(f_NL(f_N(P))) with toggles delta_N, delta_NL,
 * delta_ACT).  0 is the paper's method: normalise by the class maximum, square,
 * then the disk-mask entropy.  The low bits switch a step off; bits 4..7 pick
 * the activation that replaces the entropy. */
#define VSAOGM_MODE_NO_NORM 1u        /* skip f_N (division by max P)        */
#define VSAOGM_MODE_NO_SQUARE 2u      /* skip f_NL (squaring)                */
#define VSAOGM_ACT_ENTROPY (0u << 4)  /* Algorithm 2 (default)               */
#define VSAOGM_ACT_RELU (1u << 4)     /* max(0, x) per cell                  */
#define VSAOGM_ACT_TANH (2u << 4)     /* tanh(x) per cell                    */
#define VSAOGM_ACT_SIGMOID (3u << 4)  /* 1 / (1 + e^-x) per cell             */
#define VSAOGM_ACT_NONE (4u << 4)     /* identity (delta_ACT = 0)            */
#define VSAOGM_ACT_MASK (15u << 4)

/* vsaogm_config.flags */
#define VSAOGM_FLAG_CHECKED 1u /* encode synchronises and reports rejected points */
#define VSAOGM_FLAG_ATOMIC 2u  /* bundle with atomics (no partial-sum scratch,
                                  result not bitwise reproducible)             */
#define VSAOGM_FLAG_WINDOW_MAP_MAX 4u /* window queries normalise by the maxima of
                                  the whole map (Eq. non-linearities, Fig. 2E),
                                  so a window equals the same cells of
                                  vsaogm_query; see vsaogm_query_window     */

/* Map parameters (Sec. III-B2 Initialization, Sec. III-B3 tiling, Table of
 * VSA-OGM parameters).  Memory per map: 2 * tiles_x * tiles_y * D * 8 bytes,
 * plus, for a tensor-core decode_prec, the decode's x-phasor table of about
 * grid_w * D * 8 bytes (half that for FP8X3), built once at creation. */
typedef struct {
    int32_t D;            /* FHRR dimension (complex elements per memory), >= 1 */
    int32_t grid_w;       /* cells along x, >= 1                                  */
    int32_t grid_h;       /* cells along y, >= 1                                  */
    float resolution;     /* cell edge in metres, > 0                             */
    float x_min, y_min;   /* lower-left corner of the map in metres               */
    int32_t tiles_x;      /* delta along x (evenly sized tiles), >= 1             */
    int32_t tiles_y;      /* delta along y, >= 1; tiles_x * tiles_y <= 1024       */
    float length_scale;   /* l of Eq. fb-with-ls-1d in metres, > 0                */
    int32_t r_occ;        /* disk radius r(psi = 1) in cells, 0..16              */
    int32_t r_emp;        /* disk radius r(psi = 0) in cells, 0..16              */
    float rho;            /* decision threshold of Eq. classification             */
    uint64_t seed;        /* SplitMix64 seed of the axis frequencies              */
    int32_t decode_prec;  /* VSAOGM_DECODE_*                                      */
    uint32_t flags;       /* VSAOGM_FLAG_*                                        */
    uint32_t decode_mode; /* VSAOGM_MODE_* | VSAOGM_ACT_*; 0 = the paper's method  */
} vsaogm_config;

typedef struct vsaogm_map vsaogm_map;

/* Fills *cfg with defaults: D 8192, 400 x 400 cells of 0.1 m from (-20, -20),
 * 4 x 4 tiles, l = 0.1 m, r_occ = r_emp = 3, rho = 0, seed 0, FP32 decode.
 * The radii follow the ToySim and EviLOG rows of the paper's parameter table;
 * the rest is a service of the library (no counterpart in the paper). */
void vsaogm_config_default(vsaogm_config *cfg);

/* Creates a map (Sec. III-B2, III-B3): validates *cfg, draws the axis
 * frequencies and allocates zeroed memories on the current CUDA device.
 * Axis frequencies: nu_x[k] and nu_y[k] (cycles per metre, float32) are
 * f32((2u - 1) / (2 l)) with u the top 53 bits / 2^53 of SplitMix64 outputs
 * 2k and 2k + 1 for `seed`, i.e. theta = 2 pi l nu uniform on (-pi, pi).
 * Synchronous.  Errors: E_INVAL (bad config, NULL), E_NOMEM, E_CUDA.        */
int vsaogm_create(const vsaogm_config *cfg, vsaogm_map **out);

/* Frees the map and everything it owns.  Synchronises the device first.
 * NULL is accepted.
 * No counterpart in the paper: a service of the library. */
int vsaogm_destroy(vsaogm_map *map);

/* Sets every memory to zero (asynchronous on `stream`).
 * The empty memories a map starts from before Algorithm 1 bundles into it.
 * Errors: E_INVAL (NULL map), E_CUDA. */
int vsaogm_reset(vsaogm_map *map, void *stream);

/* Encoding and bundling (Eq. fb-with-ls-2d, Eq. bundling, Algorithm 1):
 * for each point p with label psi, the nearest tile centre beta is found
 * (ties go to the lower tile, points outside the map go to the nearest edge
 * tile) and phi_k(p) = exp(i 2 pi (nu_x[k] p_x + nu_y[k] p_y)) is added to
 * memory 2 beta + psi for all k < D.
 * xy_dev: float [n][2], 8-byte aligned; labels_dev: uint8 [n], values 0 or 1.  n = 0 is a
 * no-op.  Points with a label above 1 or a non-finite coordinate are not
 * bundled; they are counted (see vsaogm_rejected) and, with
 * VSAOGM_FLAG_CHECKED, the call synchronises and returns E_DATA.
 * Uses library-owned scratch that grows on demand (a growing call allocates
 * and synchronises).  Errors: E_INVAL (NULL with n > 0, n < 0), E_NOMEM,
 * E_CUDA, E_DATA.                                                           */
int vsaogm_encode_bundle(vsaogm_map *map, const float *xy_dev, const uint8_t *labels_dev,
                         int64_t n, void *stream);

/* Encoding and bundling without any allocation (the paper has no counterpart;
 * this is a service of the library).  Same inputs, outputs and result as
 * vsaogm_encode_bundle, within its tolerance, but the call never calls
 * cudaMalloc, cudaFree or any other allocating routine.  It is meant for
 * callers that must not allocate device memory: a real-time control loop, for
 * which cudaMalloc can synchronise the whole device and stall for
 * milliseconds, or a host process that runs under a fixed device-memory budget
 * owned by another allocator.  Map creation still allocates; do that at
 * set-up time.
 * Scratch lives in one static 4 MiB device array inside the library, which
 * every GPU that loads the library keeps until the process exits.  Its
 * device address is looked up (cudaGetSymbolAddress) once per device by
 * vsaogm_create, with that device current, so the call itself does no
 * lookup and loads no module.  All calls share the array and each call
 * writes every scratch word it reads, so nothing carries over between calls;
 * calls whose work overlaps on the GPU (different streams, or different maps
 * at the same time) race and give wrong results: order them on one stream.
 * Bundling adds into the memories with atomics, so the result is not bitwise
 * reproducible.  Each tile is bundled relative to its own centre (no bundling
 * patches), so points far from the centre of a wide tile take the exact phase
 * reduction.
 * Limits, both checked on the host before any GPU work (E_INVAL): n <=
 * 262144 points per call; and the sort's tables plus the sorted points must
 * fit the array: 4 B x ceil(n / 2048) x (2T + 1) for the per-block counts,
 * 16 B per chunk, 8 B per point and a few 256-byte roundings, which only
 * maps of many tiles with n near the limit can exceed.  The map's device must
 * be current.  With VSAOGM_FLAG_CHECKED the call synchronises and returns
 * E_DATA when points were rejected, as vsaogm_encode_bundle does (reading the
 * counter into host stack variables allocates nothing).  No stage timing is
 * recorded.  Errors: E_INVAL, E_CUDA, E_DATA.                               */
int vsaogm_encode_bundle_noalloc(vsaogm_map *map, const float *xy_dev,
                                 const uint8_t *labels_dev, int64_t n, void *stream);

/* Decoding (Eqs. vector-normalization, loc-query, non-linearities):
 * heat_dev (float [2][H][W]) receives P_hat(psi | cell) =
 * (P / max_map P)^2 with P = Re sum_k conj(w_k) phi_k(cell) / ||w|| for the
 * memory w of the cell's tile and class; the maximum runs over the whole map.
 * A class whose maximum is <= 0 (or whose memories are all zero) gives 0.
 * Errors: E_INVAL, E_CUDA.                                                  */
int vsaogm_decode(vsaogm_map *map, float *heat_dev, void *stream);

/* Entropy extraction, softmax, signed difference and classification
 * (Algorithm 2, Eqs. entropy-mask, softmax, psd, classification) applied to
 * P_hat from vsaogm_decode: H(psi | x, y) = -sum over in-grid cells within
 * Euclidean distance r(psi) (cells, inclusive) of P_hat ln P_hat (0 ln 0 = 0);
 * occ_dev (float [H][W]) = Pr(psi = 1); ogm_dev (float [H][W], nullable) =
 * Pr(1) - Pr(0); cls_dev (uint8 [H][W], nullable) = 1 where OGM >= rho.
 * Errors: E_INVAL, E_CUDA.                                                  */
int vsaogm_entropy(vsaogm_map *map, const float *heat_dev, float *occ_dev, float *ogm_dev,
                   uint8_t *cls_dev, void *stream);

/* Decode and entropy in one call, with the non-linearity fused into the
 * entropy pass.  heat_dev (float [2][H][W]) is caller-provided scratch that
 * receives the normalised similarity P (before the non-linearity).  Outputs
 * as vsaogm_entropy.  Errors: E_INVAL, E_CUDA.
 * Eqs. vector-normalization, loc-query and non-linearities, then Algorithm 2
 * and Eqs. softmax, psd, classification, as vsaogm_decode followed by
 * vsaogm_entropy. */
int vsaogm_query(vsaogm_map *map, float *heat_dev, float *occ_dev, float *ogm_dev,
                 uint8_t *cls_dev, void *stream);

/* Local map query for the window of cells [x0, x0 + w) x [y0, y0 + h):
 * Eqs. vector-normalization, loc-query and non-linearities, Algorithm 2 and
 * Eqs. softmax, psd, classification, restricted to a window.  The region
 * decoded is the window grown by R = max(r_occ, r_emp) cells on each side and
 * clipped to the map, so every window cell sees its whole disk; the maximum of
 * Eq. non-linearities is taken over that region (a local query normalises by
 * what it decodes; for the whole map this equals vsaogm_query).
 * With VSAOGM_FLAG_WINDOW_MAP_MAX the maximum is the whole map's, as the
 * paper defines it, and the window's outputs equal the same cells of
 * vsaogm_query: the whole map is decoded into library-owned scratch (float
 * [2][H][W], grown on first use or by vsaogm_reserve) whenever the memories
 * have changed since the last such decode (every call that writes them counts
 * as a change), and the window's entropy reads from it; heat_dev still
 * receives P of the region.  Calls on the map must then be ordered on one
 * stream, as for every call.
 * heat_dev: caller scratch of vsaogm_window_scratch() floats (receives P of
 * the region); occ_dev (float [h][w], row stride w); ogm_dev, cls_dev nullable
 * [h][w].  Errors: E_INVAL (window not inside the map, NULL), E_CUDA.       */
int vsaogm_query_window(vsaogm_map *map, int32_t x0, int32_t y0, int32_t w, int32_t h,
                        float *heat_dev, float *occ_dev, float *ogm_dev, uint8_t *cls_dev,
                        void *stream);

/* Decoded map of the window of cells [x0, x0 + w) x [y0, y0 + h): Eqs.
 * vector-normalization, loc-query and non-linearities restricted to the
 * window.  heat_dev (float [2][h][w], row stride w) receives P_hat of both
 * classes.  The maximum of Eq. non-linearities is the window's own (a local
 * decode normalises by what it decodes; for the whole map this equals
 * vsaogm_decode), or, with VSAOGM_FLAG_WINDOW_MAP_MAX, the whole map's, as the
 * paper defines it: the whole map is then decoded into library-owned scratch
 * as vsaogm_query_window does, and the window's cells equal the same cells of
 * vsaogm_decode.  Errors: E_INVAL (window not inside the map, NULL), E_CUDA.  */
int vsaogm_decode_window(vsaogm_map *map, int32_t x0, int32_t y0, int32_t w, int32_t h,
                         float *heat_dev, void *stream);

/* Floats of heat scratch vsaogm_query_window needs for that window.
 * No counterpart in the paper: a service of the library.
 * Errors: E_INVAL (NULL, window not inside the map). */
int vsaogm_window_scratch(const vsaogm_map *map, int32_t x0, int32_t y0, int32_t w, int32_t h,
                          int64_t *floats);

/* End-to-end call on host buffers: copies xy_host/labels_host to the device,
 * bundles them, runs vsaogm_query and copies Pr(psi = 1) back into occ_host
 * (float [H][W]); returns after the stream has finished.  Device staging is
 * owned by the map and grows on demand.  Errors: as the calls it makes.
 * The whole method (Algorithm 1, then the decoding and Algorithm 2) on host
 * buffers. */
int vsaogm_update_query_host(vsaogm_map *map, const float *xy_host, const uint8_t *labels_host,
                             int64_t n, float *occ_host, void *stream);

/* Grows the map's scratch up front so that later calls allocate nothing:
 * vsaogm_encode_bundle with up to max_points points per call, and every
 * vsaogm_decode / vsaogm_query / vsaogm_query_window.  For servers that must
 * not allocate (cudaMalloc synchronises the device) once they serve requests.
 * Synchronous.  Errors: E_INVAL, E_NOMEM, E_CUDA.
 * No counterpart in the paper: a service of the library. */
int vsaogm_reserve(vsaogm_map *map, int64_t max_points);

/* Number of points rejected by vsaogm_encode_bundle since the last reset
 * (synchronises `stream`).
 * No counterpart in the paper: a service of the library.
 * Errors: E_INVAL (NULL), E_CUDA. */
int vsaogm_rejected(vsaogm_map *map, int64_t *count, void *stream);

/* Synchronises `stream` and reports device-side failures recorded since the
 * last call: E_TIMEOUT if a kernel gave up on a bounded wait (its outputs are
 * then invalid), else VSAOGM_OK.  Clears the record.
 * No counterpart in the paper: a service of the library. */
int vsaogm_status(vsaogm_map *map, void *stream);

/* Copies the memories (complex64 [2T][D], tile-centred frame) to omega_dev.
 * Checkpoint: the memories with the configuration and seed are the map's whole
 * state (the model whose size the paper reports); the call itself has no
 * counterpart in the paper.
 * Errors: E_INVAL (NULL), E_CUDA. */
int vsaogm_get_memory(const vsaogm_map *map, float *omega_dev, void *stream);

/* Replaces the memories with omega_dev (complex64 [2T][D]).
 * Resume from a checkpoint (see vsaogm_get_memory); no counterpart in the
 * paper as a call.
 * Errors: E_INVAL (NULL), E_CUDA. */
int vsaogm_set_memory(vsaogm_map *map, const float *omega_dev, void *stream);

/* Multi-map fusion (Algorithm 3): adds src's memories into dst's.  Both maps
 * must share the axis vectors (D, seed, length scale), the tiling and the
 * grid; otherwise E_INVAL.  Maps must be on the same device.              */
int vsaogm_fuse(vsaogm_map *dst, const vsaogm_map *src, void *stream);

/* Copies the axis frequencies (cycles per metre) into host arrays of D floats.
 * The axis vectors of Sec. III-B2, as frequencies.
 * Errors: E_INVAL (NULL). */
int vsaogm_get_axis_frequencies(const vsaogm_map *map, float *nu_x_host, float *nu_y_host);

/* Geometry of the map: number of tiles and memories.
 * delta_x * delta_y tiles and two memories per tile (Sec. III-B3).
 * Errors: E_INVAL (NULL map). */
int vsaogm_get_shape(const vsaogm_map *map, int32_t *n_tiles, int32_t *n_memories);

/* Stage timing (tracing).  Stages of the calls above, in order: */
#define VSAOGM_STAGE_SORT 0      /* tile assignment + counting sort (1-4 kernels)*/
#define VSAOGM_STAGE_ENCODE 1    /* FHRR encode + bundle of the chunks           */
#define VSAOGM_STAGE_REDUCE 2    /* fixed-order sum of partial memories          */
#define VSAOGM_STAGE_NORMS 3     /* memory norms (Eq. vector-normalization)      */
#define VSAOGM_STAGE_DECODE 4    /* similarity contraction (Eq. loc-query) + max */
#define VSAOGM_STAGE_NONLINEAR 5 /* (P / max P)^2 in place (vsaogm_decode only)  */
#define VSAOGM_STAGE_ENTROPY 6   /* entropy stencil + softmax + PSD + threshold  */
#define VSAOGM_N_STAGES 7

/* Turns stage timing on or off for `map`.  When on, each stage is bracketed
 * by two CUDA events recorded on the call's stream (a few microseconds of
 * overhead per stage).  Kernel launches are counted whether timing is on or
 * not.  Errors: E_INVAL, E_CUDA.
 * No counterpart in the paper: a service of the library. */
int vsaogm_set_timing(vsaogm_map *map, int enable);

/* Accumulated device milliseconds (ms[VSAOGM_N_STAGES], nullable) and kernel
 * launch counts (launches[VSAOGM_N_STAGES], nullable) per stage since the last
 * reset; resets the counters when `reset` is non-zero.  Synchronises with
 * every stream the timed calls used.  Errors: E_INVAL, E_CUDA.
 * No counterpart in the paper: a service of the library. */
int vsaogm_stage_times(vsaogm_map *map, double *ms, int64_t *launches, int reset);

/* Batches: many maps in one step.  The paper runs one map per call; a batch
 * runs the same stages (Algorithm 1 and Sec. III-B4 encode + bundle, then
 * Eqs. vector-normalization and loc-query, the non-linearities, Algorithm 2
 * and Eqs. softmax, psd, classification) for up to VSAOGM_MAX_BATCH maps with
 * one kernel launch per stage across all maps, so that small maps share the
 * GPU instead of each leaving most SMs idle.  Results equal those of
 * vsaogm_encode_bundle followed by vsaogm_query on each map up to the
 * summation order inside each memory (one fixed order per map shape and point
 * set: a batch is deterministic run to run) and the decode slicing.
 *  - A batch refers to its maps; they must outlive it and keep their
 *    configuration.  Every map needs decode_prec BF16X3, FP16X3 or FP8X3 (the same
 *    for all), the deterministic bundling (no VSAOGM_FLAG_ATOMIC) and one
 *    device.  The batch owns its own scratch, so per-map calls on its maps
 *    never move memory a captured step uses.
 *  - Per-map arrays (xy_dev, labels_dev, n, heat_dev, occ_dev, ogm_dev) have
 *    `count` entries, in the order of `maps`.  n[i] = 0 skips map i's encode
 *    (its query still runs).  heat_dev[i]: float [2][H_i][W_i] receiving P;
 *    occ_dev[i], ogm_dev[i] (ogm_dev or its entries nullable): float
 *    [H_i][W_i] as vsaogm_query.  `reset` non-zero clears each map's memories
 *    first (a fresh map per step); zero accumulates into them.
 *  - Steps of one batch are not thread-safe and must be ordered (one stream).
 *  - Errors: E_INVAL, E_NOMEM, E_CUDA.  Device-side timeouts are reported by
 *    vsaogm_status on the maps.                                             */
#define VSAOGM_MAX_BATCH 64
typedef struct vsaogm_batch vsaogm_batch;

/* Creates a batch over maps[0..count-1] (1 <= count <= VSAOGM_MAX_BATCH,
 * distinct maps).  Allocates a few small device buffers; per-map scratch
 * grows on the first step.
 * No counterpart in the paper: a service of the library. */
int vsaogm_batch_create(vsaogm_map *const *maps, int32_t count, vsaogm_batch **out);

/* Frees the batch (synchronises the device); the maps stay.  NULL is a no-op.
 * No counterpart in the paper: a service of the library. */
int vsaogm_batch_destroy(vsaogm_batch *batch);

/* One step on `stream`: optional reset, encode + bundle of every map's
 * points, then the query of every map.  Scratch grows on the first step and
 * whenever a step needs more (cudaMalloc synchronises the device); a step
 * that grows it also drops a captured step, whose graph held the old
 * buffers (vsaogm_batch_replay then fails with E_INVAL until the next
 * capture).
 * Per map, the same computation as the single-map calls (Algorithm 1 to
 * Algorithm 2); the batching itself has no counterpart in the paper. */
int vsaogm_batch_step(vsaogm_batch *batch, const float *const *xy_dev,
                      const uint8_t *const *labels_dev, const int64_t *n,
                      float *const *heat_dev, float *const *occ_dev, float *const *ogm_dev,
                      int32_t reset, void *stream);

/* Runs one step as vsaogm_batch_step (growing the scratch), then captures
 * the same step into a CUDA graph for vsaogm_batch_replay.  The graph keeps
 * every pointer and count given here: a replay reads the same input buffers
 * (the caller refills them in place with exactly n[i] points each; the point
 * counts and chunk sizes are part of the graph) and writes the same outputs.
 * `stream` must not be the default stream.  Stage
 * timing must be off on every map.  Replaces a previous capture.
 * No counterpart in the paper: a service of the library. */
int vsaogm_batch_capture(vsaogm_batch *batch, const float *const *xy_dev,
                         const uint8_t *const *labels_dev, const int64_t *n,
                         float *const *heat_dev, float *const *occ_dev,
                         float *const *ogm_dev, int32_t reset, void *stream);

/* Launches the captured step on `stream`.  E_INVAL if nothing is captured.
 * No counterpart in the paper: a service of the library. */
int vsaogm_batch_replay(vsaogm_batch *batch, void *stream);

/* Times candidate shapes of the batched step on these inputs (each a few
 * steps with reset, so the maps' memories are overwritten) and keeps the
 * fastest: the share of phasors the encode evaluates by polynomial instead
 * of the special-function unit, the encode work per persistent CTA (which
 * sets the chunk size), the decode work items per SM and how many points a
 * map must hold per bundling patch before the finer patches pay.  Synchronous.
 * Drops a captured step (capture again after tuning).  Outputs (nullable):
 * the chosen values.
 * No counterpart in the paper: a service of the library. */
int vsaogm_batch_autotune(vsaogm_batch *batch, const float *const *xy_dev,
                          const uint8_t *const *labels_dev, const int64_t *n,
                          float *const *heat_dev, float *const *occ_dev, void *stream,
                          int32_t *poly_warps, int32_t *items_per_cta, int32_t *decode_waves);

/* Stage timing of a batch (tracing): when on, vsaogm_batch_step records CUDA
 * events between its stages on the step's stream.  Stages as VSAOGM_STAGE_*:
 * SORT (with the reset), ENCODE, REDUCE, NORMS, DECODE (with the slice sums
 * and maxima) and ENTROPY (with the fused non-linearity; NONLINEAR stays 0).
 * Replays are not timed per stage; their kernels are counted.
 * No counterpart in the paper: a service of the library. */
int vsaogm_batch_set_timing(vsaogm_batch *batch, int32_t enable);

/* Accumulated milliseconds and kernel launches per stage (both nullable,
 * VSAOGM_N_STAGES entries) since the last reset; resets them when `reset` is
 * non-zero.  Synchronises with the timed steps.  Errors: E_INVAL, E_CUDA.
 * No counterpart in the paper: a service of the library. */
int vsaogm_batch_stage_times(vsaogm_batch *batch, double *ms, int64_t *launches,
                             int32_t reset);

/* Device memory the library holds right now, in bytes, over every map and
 * batch of the process (memories, tables, scratch, staging); the static
 * scratch of vsaogm_encode_bundle_noalloc is not counted.  For callers that
 * budget device memory (a server admitting maps), and to check that a failed
 * call left nothing allocated.  Every device allocation of the library is
 * counted here; with the environment variable VSAOGM_FAIL_ALLOC=n (n >= 1) set,
 * the n-th device allocation made by one call fails as if the device were out
 * of memory (a test hook for the E_NOMEM paths).
 * No counterpart in the paper: a service of the library.
 * Errors: E_INVAL (NULL). */
int vsaogm_device_bytes(int64_t *bytes);

/* Description of the last error on the calling thread ("" if none).
 * No counterpart in the paper: a service of the library. */
const char *vsaogm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VSAOGM_H */
