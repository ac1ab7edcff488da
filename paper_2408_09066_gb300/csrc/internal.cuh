// Internal declarations shared by the translation units of libvsaogm.so.
// Nothing here is part of the C ABI (include/vsaogm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <string>
#include <vector>

#include "vsaogm.h"

namespace vsaogm_impl {

// Bounds checks of the checked build (compiled with -DVSAOGM_CHECK): an access
// whose index is out of range is skipped, and the first offending source line
// is recorded in a device flag of its translation unit, which vsaogm_status
// reports as VSAOGM_E_DATA.  Guards only ever skip an access, never a barrier,
// so a failed check cannot stall a CTA.  In the normal build they vanish.
#ifdef VSAOGM_CHECK
static __device__ int g_check_line;
__device__ __forceinline__ bool check_bounds(bool ok, int line)
{
    if (!ok) atomicCAS(&g_check_line, 0, line);
    return ok;
}
#define VSAOGM_IN_BOUNDS(cond) (::vsaogm_impl::check_bounds((cond), __LINE__))
#define VSAOGM_CHECK_TU(name)                                                       \
    int take_check_line_##name()                                                    \
    {                                                                               \
        int line = 0, zero = 0;                                                     \
        if (cudaMemcpyFromSymbol(&line, g_check_line, sizeof(int)) != cudaSuccess) \
            return -1;                                                              \
        if (line) cudaMemcpyToSymbol(g_check_line, &zero, sizeof(int));             \
        return line;                                                                \
    }
#else
#define VSAOGM_IN_BOUNDS(cond) true
#define VSAOGM_CHECK_TU(name) \
    int take_check_line_##name() { return 0; }
#endif
// first out-of-range source line recorded by each translation unit since the
// last call (0: none; always 0 in the normal build)
int take_check_line_encode();
int take_check_line_decode();
int take_check_line_decode_tc();
int take_check_line_entropy();

constexpr int kMaxTiles = 1024;      // tiles_x * tiles_y
constexpr int kMaxRadius = 16;       // disk radius in cells
constexpr int kSortBlock = 2048;     // points per block of the counting sort
constexpr int kSortWarps = 8;        // warps per sort block (256 points each)
constexpr int kMaxChunk = 2048;      // points per encode chunk (upper bound)
constexpr int64_t kMaxBatch = 1 << 26;  // points per internal encode batch

// Geometry of one axis as the kernels see it.
struct AxisDev {
    int n_tiles;
    const float *bnd_lo;    // [n_tiles - 1]: largest float <= x_min + a * tile_w, a = 1..
    const float2 *centre;   // [n_tiles]: tile centres as hi + lo (hi = f32(c), lo = f32(c - hi))
};

// Patches: for bundling only, a tile too wide for the fast phase reduction is
// cut into nx x ny patches; a chunk's points are summed relative to their
// patch's centre and the chunk's partial memory is then turned into the tile
// frame by one phasor per frequency.  n = 1: the tile is its own patch.
struct PatchDev {
    int n, nx, ny;              // patches per tile (n = nx ny), along x and along y
    float hw_x, hw_y;           // tile half extents, metres
    float inv_pw_x, inv_pw_y;   // patches per metre along x and y
    const float *cx, *cy;       // [nx], [ny]: patch centres relative to the tile centre
};

// Cell table of one axis: the tile of each cell (Algorithm 1's rule applied to
// the cell centre) and the cell centre relative to that tile's centre.
struct CellAxisDev {
    const int *tile;        // [cells]
    const float *offset;    // [cells] f32(cell centre - tile centre), metres
};

// One CTA's worth of decode work: a block of cells inside one tile.
struct DecodeBlock {
    int tile;       // beta
    int i0, j0;     // first column / row of the block
    int i1, j1;     // one past the last column / row (clipped to the tile)
};

// Blocks of one decode launch, passed by value as a kernel parameter.
constexpr int kMaxLaunchBlocks = 128;
// Tile rows one tensor-core decode block may span (its rows cross tile rows;
// DecodeBlock.tile is then the tile column).
constexpr int kMaxBlockTiles = 16;
// Frequencies one tensor-core CTA accumulates in tensor memory.  The MMA's
// FP32 accumulation is not correctly rounded (its error grows about linearly
// with the number of MMAs summed into one accumulator: 1e-4 of max P after
// all 8192 frequencies of a map), so longer sums are cut into slices that the
// slice sum adds in FP32 with round-to-nearest.
constexpr int kTcMaxKPerSplit = 2048;
struct BlockBatch {
    int n;
    DecodeBlock b[kMaxLaunchBlocks];
};

// A rectangle of cells [x0, x1) x [y0, y1) of the map.
struct Region {
    int x0, y0, x1, y1;
    __host__ __device__ int w() const { return x1 - x0; }
    __host__ __device__ int h() const { return y1 - y0; }
};

// Where decode writes cell (i, j): at (i - ox, j - oy) of an OW x OH grid.
struct OutGeom {
    int ox, oy, OW, OH;
};

// Tables of the batched (many-map) kernels, passed as __grid_constant__ params.
constexpr int kMaxBatchMaps = 64;
struct BatchSortMap {
    const float2 *xy;       // points of this map's step
    const uint8_t *lab;
    int n, S, chunk;        // points, segments (memories x patches), chunk length
    AxisDev ax, ay;
    PatchDev pt;
    int *hist;              // [nb][S + 1]
    int *meta;              // seg_meta layout of Scratch
    int4 *chunks;
    float2 *sorted;
    unsigned long long *rejected;
    int nb, blk_begin;      // sort blocks of this map, its first in the launch
    int seg_begin;          // first scan CTA (group of segment columns) of this map
};
struct BatchSortTable {
    int n_maps;
    BatchSortMap m[kMaxBatchMaps];
};
// Average chunks per memory up to which a call's chunk sums run inside the
// encode launch (above it one CTA walking a memory's chunks at the end of the
// launch costs more than the separate reduction).
constexpr int kFusedChunksPerMemory = 16;

// The bundling's fixed-order chunk sums, fused into the encode: the last CTA
// to finish a (memory, frequency slice) adds that memory's chunk partials for
// the slice to the memory, in chunk order.
struct TailSum {
    const int *cbeg;        // first chunk of each segment [S patches + 1]
    unsigned *cnt;          // [memories][n_slices] finished chunks (zero between calls);
                            // null: the map's chunks are summed by reduce_batch_kernel
    float2 *omega;          // the map's memories
    int n_slices;
};
struct BatchEncodeMap {
    const float2 *pts;      // sorted tile-centred points
    const int4 *chunks;     // chunk table
    const int *n_chunks;    // device count of chunks
    const float *nu;        // [2][D]
    float2 *out;            // partial memories [chunks][D]
    long long item_begin;   // first work item of this map
    int D, slices;
    float nu_max_x, nu_max_y;
    PatchDev pt;
    int poly_warps;         // this map's warps with one polynomial frequency pair
    TailSum tail;
};
struct BatchEncodeTable {
    int n_maps, poly_warps;
    long long total;        // work items over all maps
    BatchEncodeMap m[kMaxBatchMaps];
};

struct BatchReduceMap {
    const float2 *partial;
    const int *cbeg;        // chunk range of each segment [S patches + 1]
    float2 *omega;
    int D, seg_begin;       // first global memory of this map
    int patches;            // segments (patches) per memory
};
struct BatchReduceTable {
    int n_maps, total_segs;
    BatchReduceMap m[kMaxBatchMaps];
};

struct BatchDecodeMap {
    const float2 *omega;
    const float *inv_norm, *nu, *col_off, *row_off;
    const float2 *rot;      // [2][D]: x then y phasor of a producer row step
    const int *row_tile;    // tile row of each cell row
    float *partial;         // [slices][2][H][W]
    int *status;
    int D, k_per_split, W, H, tiles_x;
    float u_scale;
    uint64_t debug_wait_ns;  // the failure-test wait limit (0: off)
    const uint8_t *xtmap;    // TMA tensor maps of the x-phasor table (hi, lo)
};
struct BatchDecodeTable {
    int n_maps;
    BatchDecodeMap m[kMaxBatchMaps];
};
struct BatchDecodeItem {
    int map, split;
    DecodeBlock b;
};
struct BatchNormMap {
    const float2 *omega;
    float *inv_norm;
    int D, mem_begin;       // first global memory of this map
};
struct BatchNormTable {
    int n_maps;
    BatchNormMap m[kMaxBatchMaps];
};
// Per-map slice sums / entropy of a batch.
struct BatchMapOut {
    const float *partial;   // decode slices
    float *heat;            // [2][H][W] P
    unsigned *maxima;
    float *occ, *ogm;       // [H][W]
    int splits, W, H;
    float inv_scale, rho;
    int r[2];               // disk radius of class 0 (empty) and 1 (occupied)
    unsigned mode;
    int blk_begin;          // first 32 x 32 entropy block of this map in the batch
    int sum_begin;          // first slice-sum block of this map in the batch
};
struct BatchOutTable {
    int n_maps;
    BatchMapOut m[kMaxBatchMaps];
};

// Grow-on-demand device buffer owned by a map.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct Scratch {
    DevBuf blk_hist;     // int [nb][S + 1] histogram, then in-place column offsets
    DevBuf seg_meta;     // int: seg_total[S+1], seg_base[S+2], chunk_begin[S+1], n_chunks[1]
    DevBuf chunks;       // int4 [max_chunks]: (segment, begin, end, 0)
    DevBuf sorted;       // float2 [n]: tile-centred coordinates sorted by segment
    DevBuf partial;      // float2 [max_chunks][D]: per-chunk partial memories
    DevBuf stage_xy;     // host-entry staging: float [n][2]
    DevBuf stage_lab;    // uint8 [n]
    DevBuf stage_heat;   // float [2][H][W]
    DevBuf stage_occ;    // float [H][W]
    DevBuf dec_partial;  // float [slices][2][H][W]: tensor-core decode partial maps
    DevBuf map_heat;     // float [2][H][W]: P of the whole map for map-max window queries
};

// CUDA-event timing of the stages of each call (tracing) and launch counts.
struct StageTimer {
    bool enabled = false;
    std::vector<cudaEvent_t> free_events;
    struct Pending {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    double ms[VSAOGM_N_STAGES] = {};
    long long launches[VSAOGM_N_STAGES] = {};
};

}  // namespace vsaogm_impl

struct vsaogm_map {
    vsaogm_config cfg;
    int device;
    int T, S;                    // tiles, memories (2T)
    double tile_w, tile_h;
    // device state owned by the map
    float *nu;                   // [2][D]: nu_x then nu_y, cycles per metre
    float nu_max[2];             // max_k |nu_x[k]|, max_k |nu_y[k]|
    int encode_packed;           // 1: f32x2 encode kernel, 0: scalar kernel
    int encode_poly_pairs;       // frequency pairs per thread on the FMA-pipe polynomial
    int encode_poly_warps;       // > 0: only this many warps per CTA use one polynomial pair
    float2 *omega;               // [S][D]
    float *inv_norm;             // [S]: 1 / ||omega||, 0 for an all-zero memory
    unsigned *maxima;            // [2]: order-preserving encoding of max P per class
    unsigned long long *rejected;  // [1]: points rejected by encode since reset
    float *bnd_x_lo, *bnd_y_lo;  // [tiles - 1]
    float2 *centre_x, *centre_y; // [tiles]: tile centres as float pairs hi + lo
    int *col_tile, *row_tile;    // [W], [H]
    float *col_off, *row_off;    // [W], [H]
    unsigned *enc_cnt;           // [S][ceil(D / 512)]: the encode's finished-chunk counters
    float2 *tc_rot;              // tensor-core decode: [2][D] phasors of a producer row step
    uint32_t *tc_xtab;           // tensor-core decode: x-phasor table, hi and lo planes [W][Dp]
    uint8_t *tc_xtmap;           // tensor-core decode: the table's two TMA tensor maps (device)
    // failure test (VSAOGM_DEBUG_WAIT_NS at creation; 0: off): the tensor-core
    // decode's pipeline waits give up after this many nanoseconds and its
    // loader warp first stalls for four times as long, so that they do
    uint64_t debug_wait_ns;
    // generation of the memories (bumped by every call that writes them) and
    // the generation whose whole-map P ws.map_heat holds (~0: none)
    uint64_t mem_gen, map_heat_gen;
    // bundling patches: [0] coarse (phases below 32 turns), [1] fine (below 4
    // turns); device tables of patch centres below
    vsaogm_impl::PatchDev patches[2];
    float *patch_cx[2], *patch_cy[2];
    std::vector<int> tile_first[2], tile_last[2];  // per axis (x, y): cells of each tile
    int *status;                           // first error code recorded by a kernel
    int r_hw[2][2 * vsaogm_impl::kMaxRadius + 1];  // disk half-widths per class and dy
    vsaogm_impl::Scratch ws;
    vsaogm_impl::StageTimer timer;
    float *host_nu;              // [2][D] host copy
};

namespace vsaogm_impl {

// Every device allocation of the library goes through dev_malloc / dev_free,
// which keep count of the bytes held (vsaogm_device_bytes).  Test hook: with
// VSAOGM_FAIL_ALLOC=n (n >= 1) in the environment, the n-th device allocation
// made since the calling entry point began (alloc_scope_begin) fails as if the
// device were out of memory, without calling cudaMalloc.
cudaError_t dev_malloc(void **p, size_t bytes);
cudaError_t dev_free(void *p);
void alloc_scope_begin();
long long device_bytes_held();

// Error reporting (thread-local message; see vsaogm_last_error).
int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);
int ensure(DevBuf &b, size_t bytes);
void free_scratch(Scratch &ws);

// Brackets one stage: records a start event on `st` when timing is on and,
// on end(), the stop event and `kernels` launches for the stage.
class StageScope {
  public:
    StageScope(vsaogm_map *m, int stage, cudaStream_t st);
    void end(int kernels);
    ~StageScope();

  private:
    vsaogm_map *m_;
    int stage_;
    cudaStream_t st_;
    cudaEvent_t a_ = nullptr;
    bool done_ = false;
};

inline AxisDev axis_x(const vsaogm_map *m) { return {m->cfg.tiles_x, m->bnd_x_lo, m->centre_x}; }
inline AxisDev axis_y(const vsaogm_map *m) { return {m->cfg.tiles_y, m->bnd_y_lo, m->centre_y}; }

// encode.cu
int encode_bundle(vsaogm_map *m, const float *xy, const uint8_t *lab, int64_t n, cudaStream_t st);
// Device address of the allocation-free encode's static scratch on `device`
// (which must be current); looked up once per device and cached.
int noalloc_scratch(int device, unsigned char **out);
int reserve_encode(vsaogm_map *m, int64_t n);
// decode.cu
int reserve_decode(vsaogm_map *m);

// decode.cu
inline Region full_region(const vsaogm_map *m);
// Blocks of at most bi x bj cells covering region r, never straddling a tile.
void region_blocks(const vsaogm_map *m, Region r, int bi, int bj, std::vector<DecodeBlock> &out);
// P over region r into heat [2][r.h()][r.w()], and the maxima over r
int decode_region(vsaogm_map *m, Region r, float *heat, cudaStream_t st);
inline int decode_raw(vsaogm_map *m, float *heat, cudaStream_t st);
int apply_nonlinearity(vsaogm_map *m, float *heat, cudaStream_t st,
                       size_t cells = 0);  // P -> P_hat in place ([2][cells]; 0: the map)
int memory_norms(vsaogm_map *m, cudaStream_t st);
// heat = inv_scale * sum over `splits` partial maps [splits][2][cells], plus maxima
int sum_slices(vsaogm_map *m, const float *partial, int splits, size_t cells, float inv_scale,
               float *heat, cudaStream_t st);
// decode_tc.cu: split-precision tensor-core decode of region r (P and maxima)
int decode_tensor_cores(vsaogm_map *m, Region r, float *heat, cudaStream_t st);
// the tensor-core decode's blocks of region r (rows across tile rows)
void tc_blocks(const vsaogm_map *m, Region r, std::vector<DecodeBlock> &out);
// builds m's tensor-core decode tables (at creation, for a tensor-core decode_prec)
int build_tc_tables(vsaogm_map *m);

// entropy.cu
// heat holds the class maps of region r ([2][r.h()][r.w()]); the outputs cover
// window win (inside r), row stride win.w().  raw_input: heat holds P and the
// non-linearity is applied on load with the map's maxima; else it holds P_hat.
int entropy(vsaogm_map *m, const float *heat, Region r, Region win, bool raw_input, float *occ,
            float *ogm, uint8_t *cls, cudaStream_t st);

// misc kernels (decode.cu)
int add_memories(float2 *dst, const float2 *src, int64_t count, cudaStream_t st);

// The patching for a call of n points: the fine one when its segments hold
// enough points each to pay for their fixed costs, else the coarse one.
const PatchDev &choose_patches(const vsaogm_map *m, int64_t n, int min_per_segment = 512);
// Whether every point inside the map lies within 4 turns of its patch centre
// under patching pt (the encode's cheapest phase path).
bool patches_near(const vsaogm_map *m, const PatchDev &pt);

// batched (many-map) stages, used by batch.cu; `ws` is scratch the batch owns
// (not the map's), so per-map calls never move memory a captured step uses
// sizes map m's sort scratch in ws for n points and fills its sort entry
// (blk_begin and seg_begin are left to the caller)
int batch_sort_entry(vsaogm_map *m, Scratch &ws, const PatchDev &pt, const float *xy,
                     const uint8_t *lab, int n, int chunk, BatchSortMap *e, int *max_chunks);
// the four sort kernels over every entry, one launch each; blocks = sum of nb,
// segs = sum of sort_scan_ctas(S + 1), max_s1 = the largest S + 1
int launch_sort_batch(const BatchSortTable &tab, int blocks, int segs, int max_s1,
                      cudaStream_t st);
// CTAs of the segment scan for S1 segment columns
int sort_scan_ctas(int S1);
// whether a call of n points over S1 - 1 segments sorts in one CTA, and that
// sort for every entry of a table (one CTA each; max_s1 the largest S + 1)
bool sort_small(int n, int S1);
int launch_sort_small_batch(const BatchSortTable &tab, int max_s1, cudaStream_t st);
void batch_encode_entry(const vsaogm_map *m, const Scratch &ws, const PatchDev &pt,
                        BatchEncodeMap *e);
int encode_batch_ctas();
int launch_encode_batch(const BatchEncodeTable &tab, unsigned long long *counter, int ctas,
                        cudaStream_t st);
// the fixed-order chunk sums of the maps whose encode entry has no fused sums
void batch_reduce_entry(const vsaogm_map *m, const Scratch &ws, const PatchDev &pt,
                        BatchReduceMap *e);
int launch_reduce_batch(const BatchReduceTable &tab, int d_max, cudaStream_t st);
int launch_norms_batch(const BatchNormTable &tab, int total_memories, cudaStream_t st);
// slice sums + maxima of every map; sum_begin numbers kSumBlockOutputs-output
// blocks over the maps, total_blocks of them
constexpr int kSumBlockOutputs = 2048;
int launch_sums_batch(const BatchOutTable &tab, int total_blocks, cudaStream_t st);
int launch_decode_tc_batch(const BatchDecodeTable &tab, const BatchDecodeItem *items,
                           int n_items, int decode_prec, cudaStream_t st);
// frequencies per tensor-core stage for a decode_prec (slices are multiples of it)
int tc_stage_freqs(int decode_prec);
int launch_entropy_batch(const BatchOutTable &tab, cudaStream_t st);
float tc_u_scale(const vsaogm_map *m);

inline Region full_region(const vsaogm_map *m)
{
    return Region{0, 0, m->cfg.grid_w, m->cfg.grid_h};
}
inline int decode_raw(vsaogm_map *m, float *heat, cudaStream_t st)
{
    return decode_region(m, full_region(m), heat, st);
}

// Order-preserving map from float to unsigned (for atomicMax of floats).
__host__ __device__ inline unsigned float_to_ordered(float f)
{
    unsigned u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(f);
#else
    memcpy(&u, &f, 4);
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float ordered_to_float(unsigned o)
{
    unsigned u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    float f;
#ifdef __CUDA_ARCH__
    f = __uint_as_float(u);
#else
    memcpy(&f, &u, 4);
#endif
    return f;
}

}  // namespace vsaogm_impl
