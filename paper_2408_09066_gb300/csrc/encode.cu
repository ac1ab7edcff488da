// Encoding and bundling (Eq. fb-with-ls-2d, Eq. bundling, Algorithm 1).
//
// Pipeline for one batch of n points (all kernels on the caller's stream):
//   1. seg_count    : segment s = 2 beta + psi of every point (Algorithm 1's
//                     nearest tile centre, exact float compares against the
//                     tile boundaries), per-block histograms.
//   2. seg_scan     : per-segment exclusive scan of the block histograms.
//   3. seg_meta     : segment bases and the chunk table (chunks of at most
//                     `chunk` points that never straddle a segment).
//   4. seg_scatter  : stable scatter of the points into segment order, in the
//                     tile-centred frame (offsets from float-pair centres with
//                     compensated FP32 differences, within an ulp).
//   5. encode_chunk : one CTA per (chunk, slice of k); each thread keeps KPT
//                     frequencies in registers, walks the chunk's points from
//                     shared memory and accumulates exp(i 2 pi nu . p) with
//                     MUFU sin/cos (or a polynomial on the FMA pipe) of the
//                     phase, reduced to [-1/2, 1/2] turns unless it stays
//                     below 4 turns.  Points are taken relative to the centre
//                     of their bundling patch, and each chunk's sum is turned
//                     into the tile frame afterwards.  Partial memories go to
//                     scratch ...
//   6. reduce       : ... and are summed per segment in a fixed order, so the
//                     result does not depend on scheduling.  With
//                     VSAOGM_FLAG_ATOMIC step 5 adds into the memories with
//                     atomics instead and step 6 is skipped.
#include <algorithm>
#include <mutex>

#include "internal.cuh"
#include "sm100.cuh"

// Scratch of vsaogm_encode_bundle_noalloc: a fixed device array, so that the
// call needs no allocation.  Every device that loads the library holds it
// until the process exits.  In host code this name is only a stand-in for the
// array; kernels receive the device address obtained with
// cudaGetSymbolAddress (see noalloc_scratch below).
static constexpr size_t kNoAllocScratchBytes = 4u << 20;  // 4 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace vsaogm_impl {
namespace {

constexpr int kScanThreads = 1024;

// Number of boundaries strictly below x (boundaries ascending): the tile index
// along one axis.  Equal to a boundary -> the lower tile (Algorithm 1's first
// minimum); beyond the map -> the edge tile (nearest centre).
__device__ __forceinline__ int tile_along(const float *bnd, int nb, float x)
{
    int lo = 0, hi = nb;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (x > bnd[mid]) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Segment (2 beta + psi) pt.n + patch, or S for a point that is rejected.
// The patch is the one containing the point's offset from its tile centre
// (clamped to the tile's edge patches; any deterministic rule would do, since
// a patch only groups points for summation).
__device__ __forceinline__ int point_segment(float x, float y, unsigned lab, const AxisDev &ax,
                                             const AxisDev &ay, const PatchDev &pt, int S)
{
    if (lab > 1u || !isfinite(x) || !isfinite(y)) return S;
    int bx = tile_along(ax.bnd_lo, ax.n_tiles - 1, x);
    int by = tile_along(ay.bnd_lo, ay.n_tiles - 1, y);
    const int mem = 2 * (by * ax.n_tiles + bx) + (int)lab;
    if (pt.n == 1) return mem;
    const float ux = (x - ax.centre[bx].x + pt.hw_x) * pt.inv_pw_x;
    const float uy = (y - ay.centre[by].x + pt.hw_y) * pt.inv_pw_y;
    const int px = (int)floorf(fminf(fmaxf(ux, 0.f), (float)(pt.nx - 1)));
    const int py = (int)floorf(fminf(fmaxf(uy, 0.f), (float)(pt.ny - 1)));
    return mem * pt.n + py * pt.nx + px;
}

// Multiplies (re, im) by exp(i 2 pi (nu_x cx + nu_y cy)): the phasor that turns a
// partial memory summed relative to a patch centre (cx, cy) into the tile's
// frame.  The phase is reduced exactly (each product against its own nearest
// integer with one FMA, as in the exact point reduction).
__device__ __forceinline__ void patch_rotate(float nux, float nuy, float cx, float cy, float &re,
                                             float &im)
{
    const float kM = 12582912.0f;
    const float p1 = __fmul_rn(nux, cx), p2 = __fmul_rn(nuy, cy);
    const float n1 = __fsub_rn(kM, __fadd_rn(p1, kM)), n2 = __fsub_rn(kM, __fadd_rn(p2, kM));
    const float g = __fadd_rn(fmaf(nux, cx, n1), fmaf(nuy, cy, n2));
    const float f = __fsub_rn(g, __fsub_rn(__fadd_rn(g, kM), kM));
    float sn, cs;
    __sincosf(__fmul_rn(f, 6.28318530717958647692f), &sn, &cs);
    const float r = re * cs - im * sn;
    im = re * sn + im * cs;
    re = r;
}

// Block-wide exclusive scan of v over kScanThreads threads; returns the prefix
// and writes the block total to *total.
__device__ int block_exclusive_scan(int v, int *total)
{
    __shared__ int warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;  // inclusive prefix over warps
    }
    __syncthreads();
    int before = (warp > 0 ? warp_sums[warp - 1] : 0) + x - v;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

// 1. Per-block histogram over segments 0..S (S = rejected) of sort block blk.
__device__ __forceinline__ void seg_count_body(const float2 *__restrict__ xy,
                                               const uint8_t *__restrict__ lab, int n,
                                               const AxisDev &ax, const AxisDev &ay,
                                               const PatchDev &pt, int S, int *__restrict__ hist,
                                               int blk, int *cnt)
{
    const int S1 = S + 1;
    for (int s = threadIdx.x; s < S1; s += blockDim.x) cnt[s] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = blk * kSortBlock + warp * (kSortBlock / kSortWarps);
    for (int r = 0; r < kSortBlock / kSortWarps / 32; ++r) {
        int i = base + r * 32 + lane;
        int seg = -1;
        if (i < n) {
            float2 p = xy[i];
            seg = point_segment(p.x, p.y, lab[i], ax, ay, pt, S);
        }
        unsigned peers = __match_any_sync(0xffffffffu, seg);
        if (seg >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[seg], __popc(peers));
    }
    __syncthreads();
    for (int s = threadIdx.x; s < S1; s += blockDim.x) hist[(size_t)blk * S1 + s] = cnt[s];
}

__global__ void __launch_bounds__(256) seg_count_kernel(const float2 *__restrict__ xy,
                                                        const uint8_t *__restrict__ lab, int n,
                                                        AxisDev ax, AxisDev ay, PatchDev pt,
                                                        int S, int *__restrict__ hist)
{
    extern __shared__ int cnt[];  // [S + 1]
    seg_count_body(xy, lab, n, ax, ay, pt, S, hist, blockIdx.x, cnt);
}

// 2. Column s of hist [nb][S1] -> exclusive prefix over blocks (in place);
//    total[s] = column sum.
// Columns cg * kScanCols .. + kScanCols - 1 of hist [nb][S1] by one CTA of
// kScanWarps warps: lane = column (coalesced rows), warp w = a contiguous run
// of block rows.  Pass 1 sums each warp's run, the runs' sums are scanned
// across warps, and pass 2 rewrites the run in place as exclusive prefixes.
constexpr int kScanCols = 32;
constexpr int kScanWarps = 32;
__device__ __forceinline__ void seg_scan_body(int *__restrict__ hist, int nb, int S1,
                                              int *__restrict__ total, int cg)
{
    __shared__ int wsum[kScanWarps][kScanCols + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = cg * kScanCols + lane;
    const bool col = s < S1;
    const int per = (nb + kScanWarps - 1) / kScanWarps;
    const int b0 = min(nb, warp * per), b1 = min(nb, b0 + per);
    // both passes read eight rows ahead into registers, so that eight loads are
    // in flight per thread (pass 2's stores would otherwise hold back each next load)
    constexpr int kAhead = 8;
    int sum = 0;
    if (col)
        for (int b = b0; b < b1; b += kAhead) {
            int v[kAhead];
#pragma unroll
            for (int j = 0; j < kAhead; ++j) v[j] = b + j < b1 ? hist[(size_t)(b + j) * S1 + s] : 0;
#pragma unroll
            for (int j = 0; j < kAhead; ++j) sum += v[j];
        }
    wsum[warp][lane] = sum;
    __syncthreads();
    int carry = 0;
    for (int w = 0; w < warp; ++w) carry += wsum[w][lane];
    if (col) {
        for (int b = b0; b < b1; b += kAhead) {
            int v[kAhead];
#pragma unroll
            for (int j = 0; j < kAhead; ++j) v[j] = b + j < b1 ? hist[(size_t)(b + j) * S1 + s] : 0;
#pragma unroll
            for (int j = 0; j < kAhead; ++j) {
                if (b + j < b1) hist[(size_t)(b + j) * S1 + s] = carry;
                carry += v[j];
            }
        }
        if (warp == kScanWarps - 1) total[s] = carry;  // the last run ends at the column sum
    }
}

__global__ void __launch_bounds__(32 * kScanWarps) seg_scan_kernel(int *__restrict__ hist, int nb,
                                                                   int S1,
                                                                   int *__restrict__ total)
{
    seg_scan_body(hist, nb, S1, total, blockIdx.x);
}

// 3. Segment bases, chunk table, rejected count.  One CTA.
//    meta layout: total[S1] | base[S1 + 1] | chunk_begin[S + 1] | n_chunks[1]
__device__ __forceinline__ void seg_meta_body(int *__restrict__ meta, int S, int chunk,
                                              int4 *__restrict__ chunks,
                                              unsigned long long *rejected)
{
    const int S1 = S + 1;
    int *total = meta, *base = meta + S1, *cbeg = base + S1 + 1, *nch_out = cbeg + S + 1;
    // bases: exclusive scan of totals (S1 entries, in rounds of kScanThreads)
    int carry = 0;
    for (int s0 = 0; s0 < S1; s0 += kScanThreads) {
        int s = s0 + threadIdx.x;
        int v = s < S1 ? total[s] : 0, tot;
        int pre = block_exclusive_scan(v, &tot);
        if (s < S1) base[s] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) base[S1] = carry;
    // chunk counts per (non-rejected) segment
    carry = 0;
    for (int s0 = 0; s0 < S; s0 += kScanThreads) {
        int s = s0 + threadIdx.x;
        int v = s < S ? (total[s] + chunk - 1) / chunk : 0, tot;
        int pre = block_exclusive_scan(v, &tot);
        if (s < S) cbeg[s] = carry + pre;
        carry += tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        cbeg[S] = carry;
        *nch_out = carry;
        if (total[S] > 0) atomicAdd(rejected, (unsigned long long)total[S]);
    }
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        int nc = (total[s] + chunk - 1) / chunk;
        for (int c = 0; c < nc; ++c) {
            int b = base[s] + c * chunk;
            chunks[cbeg[s] + c] = make_int4(s, b, min(b + chunk, base[s] + total[s]), 0);
        }
    }
    // Launch order, in the table's spare field: entry i's .w is the chunk the
    // encode's i-th CTA (or work item) takes.  Full chunks come first, then the
    // partial ones by length, longest first (in buckets of 1/32 of the chunk
    // length), so a launch ends on its shortest chunks instead of on whichever
    // chunks the segment order puts last.  Inside a bucket the order is
    // whatever the atomics give: a chunk's partial memory goes to its own slot
    // whenever it runs, so no result depends on it.
    __shared__ int ocnt[33];
    __syncthreads();  // every entry above is written before its .w is
    if (threadIdx.x < 33) ocnt[threadIdx.x] = 0;
    __syncthreads();
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        const int nc = (total[s] + chunk - 1) / chunk;
        for (int c = 0; c < nc; ++c) {
            const int sz = min(chunk, total[s] - c * chunk);
            atomicAdd(&ocnt[sz >= chunk ? 32 : (int)((long long)sz * 32 / chunk)], 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int bk = 32; bk >= 0; --bk) {
            const int n = ocnt[bk];
            ocnt[bk] = run;
            run += n;
        }
    }
    __syncthreads();
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        const int nc = (total[s] + chunk - 1) / chunk;
        for (int c = 0; c < nc; ++c) {
            const int sz = min(chunk, total[s] - c * chunk);
            const int pos = atomicAdd(&ocnt[sz >= chunk ? 32 : (int)((long long)sz * 32 / chunk)], 1);
            chunks[pos].w = cbeg[s] + c;
        }
    }
}

__global__ void __launch_bounds__(kScanThreads) seg_meta_kernel(int *__restrict__ meta, int S,
                                                                int chunk,
                                                                int4 *__restrict__ chunks,
                                                                unsigned long long *rejected)
{
    seg_meta_body(meta, S, chunk, chunks, rejected);
}

// 4. Stable scatter into segment order, tile-centred coordinates.
// a + b as the rounded sum s and its exact error e (a + b = s + e exactly).
__device__ __forceinline__ float two_sum(float a, float b, float &e)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// x - (c.x + c.y) - d for a float x, a centre given as the float pair c and a
// float d: two exact differences and the rounded sum of their errors, within an
// ulp of the correctly rounded value (no FP64, which this GPU runs at a small
// fraction of the FP32 rate).
__device__ __forceinline__ float offset_from(float x, float2 c, float d)
{
    float e1, e2;
    const float s = two_sum(x, -c.x, e1);
    const float r = two_sum(s, -d, e2);
    return __fadd_rn(r, __fsub_rn(__fadd_rn(e1, e2), c.y));
}

__device__ __forceinline__ void seg_scatter_body(const float2 *__restrict__ xy,
                                                 const uint8_t *__restrict__ lab, int n,
                                                 const AxisDev &ax, const AxisDev &ay,
                                                 const PatchDev &pt, int S,
                                                 const int *__restrict__ blk_off,
                                                 const int *__restrict__ meta,
                                                 float2 *__restrict__ sorted, int blk, int *wcnt)
{
    // wcnt: [kSortWarps][S1]: counts, then running cursors
    const int S1 = S + 1;
    const int *seg_base = meta + S1;
    for (int s = threadIdx.x; s < kSortWarps * S1; s += blockDim.x) wcnt[s] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = blk * kSortBlock + warp * (kSortBlock / kSortWarps);
    constexpr int kRounds = kSortBlock / kSortWarps / 32;
    int *mine = wcnt + warp * S1;
    // pass 1: per-warp counts (only this warp touches its row); the points and
    // their segments stay in registers for pass 2
    float2 p[kRounds];
    int seg[kRounds];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int i = base + r * 32 + lane;
        seg[r] = -1;
        p[r] = make_float2(0.f, 0.f);
        if (i < n) {
            p[r] = xy[i];
            seg[r] = point_segment(p[r].x, p[r].y, lab[i], ax, ay, pt, S);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, seg[r]);
        if (seg[r] >= 0 && lane == __ffs(peers) - 1) mine[seg[r]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // cursors: global position of each warp's first point of each segment
    for (int s = threadIdx.x; s < S1; s += blockDim.x) {
        int run = seg_base[s] + blk_off[(size_t)blk * S1 + s];
        for (int w = 0; w < kSortWarps; ++w) {
            int c = wcnt[w * S1 + s];
            wcnt[w * S1 + s] = run;
            run += c;
        }
    }
    __syncthreads();
    // pass 2: ranks in original order, write offsets from the tile (or patch)
    // centre
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const unsigned peers = __match_any_sync(0xffffffffu, seg[r]);
        int dst = 0;
        if (seg[r] >= 0) dst = mine[seg[r]] + __popc(peers & lt);
        __syncwarp();
        if (seg[r] >= 0 && lane == __ffs(peers) - 1) mine[seg[r]] += __popc(peers);
        __syncwarp();
        if (seg[r] >= 0 && seg[r] < S) {
            const int mem = seg[r] / pt.n, patch = seg[r] - mem * pt.n;
            const int beta = mem >> 1;
            const int bx = beta % ax.n_tiles, by = beta / ax.n_tiles;
            const float cx = pt.n > 1 ? pt.cx[patch % pt.nx] : 0.f;
            const float cy = pt.n > 1 ? pt.cy[patch / pt.nx] : 0.f;
            const float dx = offset_from(p[r].x, ax.centre[bx], cx);
            const float dy = offset_from(p[r].y, ay.centre[by], cy);
            if (VSAOGM_IN_BOUNDS(dst >= 0 && dst < n)) sorted[dst] = make_float2(dx, dy);
        }
    }
}

__global__ void __launch_bounds__(256) seg_scatter_kernel(const float2 *__restrict__ xy,
                                                          const uint8_t *__restrict__ lab, int n,
                                                          AxisDev ax, AxisDev ay, PatchDev pt,
                                                          int S, const int *__restrict__ blk_off,
                                                          const int *__restrict__ meta,
                                                          float2 *__restrict__ sorted)
{
    extern __shared__ int wcnt[];
    seg_scatter_body(xy, lab, n, ax, ay, pt, S, blk_off, meta, sorted, blockIdx.x, wcnt);
}

// 1'-4'. The four sort kernels over every map of a batch, one launch each:
//        CTA q finds its map by binary search over each map's first CTA.
__device__ __forceinline__ int batch_sort_map(const BatchSortTable &tab, int q, bool by_segment)
{
    int lo = 0, hi = tab.n_maps - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        const int first = by_segment ? tab.m[mid].seg_begin : tab.m[mid].blk_begin;
        if (first <= q) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) batch_seg_count_kernel(const __grid_constant__ BatchSortTable tab)
{
    extern __shared__ int cnt[];
    const BatchSortMap &M = tab.m[batch_sort_map(tab, blockIdx.x, false)];
    seg_count_body(M.xy, M.lab, M.n, M.ax, M.ay, M.pt, M.S, M.hist, blockIdx.x - M.blk_begin,
                   cnt);
}

__global__ void __launch_bounds__(32 * kScanWarps) batch_seg_scan_kernel(const __grid_constant__ BatchSortTable tab)
{
    const BatchSortMap &M = tab.m[batch_sort_map(tab, blockIdx.x, true)];
    seg_scan_body(M.hist, M.nb, M.S + 1, M.meta, blockIdx.x - M.seg_begin);
}

__global__ void __launch_bounds__(kScanThreads) batch_seg_meta_kernel(const __grid_constant__ BatchSortTable tab)
{
    const BatchSortMap &M = tab.m[blockIdx.x];
    seg_meta_body(M.meta, M.S, M.chunk, M.chunks, M.rejected);
}

__global__ void __launch_bounds__(256) batch_seg_scatter_kernel(const __grid_constant__ BatchSortTable tab)
{
    extern __shared__ int wcnt[];
    const BatchSortMap &M = tab.m[batch_sort_map(tab, blockIdx.x, false)];
    seg_scatter_body(M.xy, M.lab, M.n, M.ax, M.ay, M.pt, M.S, M.hist, M.meta, M.sorted,
                     blockIdx.x - M.blk_begin, wcnt);
}

// 1-4 in one CTA for a small call (n <= kSmallSortPoints points, S + 1 <=
// kSmallSortSegs segments): the same stable counting sort with the 32 warps of
// one CTA in place of the sort blocks (warp w takes points w * PW .. + PW - 1,
// in order), so a small update costs one launch instead of four.
constexpr int kSmallSortWarps = 32;
constexpr int kSmallSortPoints = 8192;
constexpr int kSmallSortSegs = 1536;  // 32 x 1536 counters: 192 KB of shared memory
__device__ __forceinline__ void seg_sort_small_body(
    const float2 *__restrict__ xy, const uint8_t *__restrict__ lab, int n, const AxisDev &ax,
    const AxisDev &ay, const PatchDev &pt, int S, int chunk, int *__restrict__ meta,
    int4 *__restrict__ chunks, unsigned long long *rejected, float2 *__restrict__ sorted,
    int *wcnt)
{
    // wcnt: [kSmallSortWarps][S1]: counts, then cursors
    const int S1 = S + 1;
    for (int i = threadIdx.x; i < kSmallSortWarps * S1; i += blockDim.x) wcnt[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pw = (n + kSmallSortWarps * 32 - 1) / (kSmallSortWarps * 32) * 32;  // points a warp
    const int base = warp * pw;
    int *mine = wcnt + warp * S1;
    for (int r = 0; r < pw; r += 32) {
        const int i = base + r + lane;
        int seg = -1;
        if (i < n) {
            const float2 p = xy[i];
            seg = point_segment(p.x, p.y, lab[i], ax, ay, pt, S);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, seg);
        if (seg >= 0 && lane == __ffs(peers) - 1) mine[seg] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per segment: the warps' exclusive offsets and the segment's total
    for (int s = threadIdx.x; s < S1; s += blockDim.x) {
        int run = 0;
        for (int w = 0; w < kSmallSortWarps; ++w) {
            const int c = wcnt[w * S1 + s];
            wcnt[w * S1 + s] = run;
            run += c;
        }
        meta[s] = run;
    }
    __syncthreads();
    seg_meta_body(meta, S, chunk, chunks, rejected);
    __syncthreads();
    const int *seg_base = meta + S1;
    for (int s = threadIdx.x; s < kSmallSortWarps * S1; s += blockDim.x)
        wcnt[s] += seg_base[s % S1];
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < pw; r += 32) {
        const int i = base + r + lane;
        int seg = -1;
        float2 p = make_float2(0.f, 0.f);
        if (i < n) {
            p = xy[i];
            seg = point_segment(p.x, p.y, lab[i], ax, ay, pt, S);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, seg);
        int dst = 0;
        if (seg >= 0) dst = mine[seg] + __popc(peers & lt);
        __syncwarp();
        if (seg >= 0 && lane == __ffs(peers) - 1) mine[seg] += __popc(peers);
        __syncwarp();
        if (seg >= 0 && seg < S) {
            const int mem = seg / pt.n, patch = seg - mem * pt.n;
            const int beta = mem >> 1;
            const int bx = beta % ax.n_tiles, by = beta / ax.n_tiles;
            const float cx = pt.n > 1 ? pt.cx[patch % pt.nx] : 0.f;
            const float cy = pt.n > 1 ? pt.cy[patch / pt.nx] : 0.f;
            const float dx = offset_from(p.x, ax.centre[bx], cx);
            const float dy = offset_from(p.y, ay.centre[by], cy);
            if (VSAOGM_IN_BOUNDS(dst >= 0 && dst < n)) sorted[dst] = make_float2(dx, dy);
        }
    }
}

__global__ void __launch_bounds__(32 * kSmallSortWarps) seg_sort_small_kernel(
    const float2 *__restrict__ xy, const uint8_t *__restrict__ lab, int n, AxisDev ax,
    AxisDev ay, PatchDev pt, int S, int chunk, int *__restrict__ meta, int4 *__restrict__ chunks,
    unsigned long long *rejected, float2 *__restrict__ sorted)
{
    extern __shared__ int wcnt[];
    seg_sort_small_body(xy, lab, n, ax, ay, pt, S, chunk, meta, chunks, rejected, sorted, wcnt);
}

// The small maps of a batch: one CTA each.
__global__ void __launch_bounds__(32 * kSmallSortWarps) batch_seg_sort_small_kernel(
    const __grid_constant__ BatchSortTable tab)
{
    extern __shared__ int wcnt[];
    const BatchSortMap &M = tab.m[blockIdx.x];
    seg_sort_small_body(M.xy, M.lab, M.n, M.ax, M.ay, M.pt, M.S, M.chunk, M.meta, M.chunks,
                        M.rejected, M.sorted, wcnt);
}

// 5. Encode + bundle one chunk of one segment over a slice of 256*KPT
//    frequencies.  The phase in turns t = nu_x dx + nu_y dy is reduced to
//    f = t - rint(t) in [-1/2, 1/2] and then one MUFU sin and one MUFU cos of
//    2 pi f are taken.
//    Fast reduction (every |nu dx|, |nu dy| of the chunk below 32 turns):
//      p1 = fl(nu_x dx), p2 = fl(nu_y dy), r = rint(p1 + p2),
//      f = fl(fl(p1 - r) + p2).  Errors: the two product roundings (at most
//      2^-20 turns each) and the rounding of p1 - r when |p1 - r| outgrows
//      |p1| (at most ulp(32.5)/2 = 2^-19 turns); about 4e-6 turns (2.5e-5
//      rad) in the worst case, far less on average.
//    Exact reduction (points far from their tile centre, e.g. large tiles or
//      points outside the map): each product is reduced against its own
//      nearest integer with one FMA, f_i = fl(nu_i d_i - rint(p_i)), whose
//      exact value is at most 1/2 + 2^-24 |p_i| in magnitude, so the FMA's
//      single rounding costs at most 2^-25 turns; g = fl(f1 + f2) (|g| <= 1,
//      another 2^-25) is reduced once more to [-1/2, 1/2] (exact).  The phase
//      error is at most 3 * 2^-25 turns (6e-7 rad).
template <int KPT, bool EXACT>
__device__ __forceinline__ void encode_points(const float2 *sp, int len, const float (&nx)[KPT],
                                              const float (&ny)[KPT], float (&ar)[KPT],
                                              float (&ai)[KPT])
{
    const float kMagic = 12582912.0f;  // 1.5 * 2^23: x + M - M = rint(x) for |x| < 2^22
    const float kTwoPi = 6.28318530717958647692f;
#pragma unroll 2
    for (int p = 0; p < len; ++p) {
        const float2 q = sp[p];
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            float p1 = __fmul_rn(nx[j], q.x);
            float p2 = __fmul_rn(ny[j], q.y);
            float f;
            if (EXACT) {
                // -rint(p) = M - (p + M), exactly
                float n1 = __fsub_rn(kMagic, __fadd_rn(p1, kMagic));
                float n2 = __fsub_rn(kMagic, __fadd_rn(p2, kMagic));
                float g = __fadd_rn(fmaf(nx[j], q.x, n1), fmaf(ny[j], q.y, n2));
                f = __fsub_rn(g, __fsub_rn(__fadd_rn(g, kMagic), kMagic));
            } else {
                float r = __fsub_rn(__fadd_rn(__fadd_rn(p1, p2), kMagic), kMagic);
                f = __fadd_rn(__fsub_rn(p1, r), p2);
            }
            float s, co;
            __sincosf(__fmul_rn(f, kTwoPi), &s, &co);
            ar[j] += co;
            ai[j] += s;
        }
    }
}

template <int KPT, bool ATOMIC>
__global__ void __launch_bounds__(256) encode_chunk_kernel(const float2 *__restrict__ pts,
                                                           const int4 *__restrict__ chunks,
                                                           const int *__restrict__ n_chunks,
                                                           const float *__restrict__ nu, int D,
                                                           float nu_max_x, float nu_max_y,
                                                           PatchDev pt, float2 *__restrict__ out)
{
    __shared__ float2 sp[kMaxChunk];
    __shared__ unsigned s_bound[2];
    const int c = blockIdx.x;
    if (c >= *n_chunks) return;
    const int4 ch = chunks[c];
    // a chunk holds at most kMaxChunk points (the staging buffer's size)
    const int len = VSAOGM_IN_BOUNDS(ch.z >= ch.y && ch.z - ch.y <= kMaxChunk) ? ch.z - ch.y : 0;
    const int kbase = blockIdx.y * (256 * KPT) + threadIdx.x;
    float nx[KPT], ny[KPT], ar[KPT], ai[KPT];
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        int k = kbase + j * 256;
        nx[j] = k < D ? nu[k] : 0.f;
        ny[j] = k < D ? nu[D + k] : 0.f;
        ar[j] = 0.f;
        ai[j] = 0.f;
    }
    if (threadIdx.x < 2) s_bound[threadIdx.x] = 0u;
    __syncthreads();
    float mx = 0.f, my = 0.f;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        float2 q = pts[ch.y + i];
        sp[i] = q;
        mx = fmaxf(mx, fabsf(q.x));
        my = fmaxf(my, fabsf(q.y));
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, o));
    }
    // non-negative floats order like their bit patterns
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&s_bound[0], __float_as_uint(mx));
        atomicMax(&s_bound[1], __float_as_uint(my));
    }
    __syncthreads();
    const bool fast = __uint_as_float(s_bound[0]) * nu_max_x < 32.0f &&
                      __uint_as_float(s_bound[1]) * nu_max_y < 32.0f;
    if (fast)
        encode_points<KPT, false>(sp, len, nx, ny, ar, ai);
    else
        encode_points<KPT, true>(sp, len, nx, ny, ar, ai);
    const int mem = ch.x / pt.n, patch = ch.x - mem * pt.n;
    if (pt.n > 1) {
        const float cx = pt.cx[patch % pt.nx], cy = pt.cy[patch / pt.nx];
#pragma unroll
        for (int j = 0; j < KPT; ++j) patch_rotate(nx[j], ny[j], cx, cy, ar[j], ai[j]);
    }
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        int k = kbase + j * 256;
        if (k < D) {
            if (ATOMIC) {
                float2 *w = out + (size_t)mem * D + k;
                atomicAdd(&w->x, ar[j]);
                atomicAdd(&w->y, ai[j]);
            } else {
                out[(size_t)c * D + k] = make_float2(ar[j], ai[j]);
            }
        }
    }
}

// 5'. The same encode + bundle with packed FP32 pairs (two frequencies per
//     instruction) and part of the unit phasors evaluated on the FMA pipe.
//     Of the NP frequency pairs a thread holds, NPOLY pairs use
//     exp(i 2 pi f) = (exp(i pi f))^2 with exp(i pi f) from polynomials on
//     |pi f| <= pi/2 (sin and cos, five coefficients each, fitted
//     near-minimax by phasor_poly.py: errors 3.3e-9 and 4.7e-8, about 1.5e-7
//     in float32), squared as a complex number; the other pairs use MUFU
//     sin/cos.  The phase reduction is the one of encode_points, lane by lane.

// TIER 0 (every |nu d| of the chunk below 4 turns): the MUFU lanes take
// sin/cos of 2 pi t without reducing t (MUFU's own argument reduction costs it
// about 1e-7 x |2 pi t| <= 5e-6 rad here, measured on GB300, less than the
// reduction's 3 operations would save); the polynomial lanes reduce t first.
// TIER 1: the fast reduction.  TIER 2: the exact reduction.
template <int NP, int NPOLY, int TIER>
__device__ __forceinline__ void encode_points_x2(const float2 *sp, int len,
                                                 const sm100::f32x2 (&nx)[NP],
                                                 const sm100::f32x2 (&ny)[NP],
                                                 sm100::f32x2 (&ac)[NP], sm100::f32x2 (&as)[NP])
{
    using namespace sm100;
    const f32x2 kM = pack2(12582912.0f, 12582912.0f);
    const f32x2 kTwoPi = pack2(6.28318530717958647692f, 6.28318530717958647692f);
    const f32x2 kPi = pack2(3.14159265358979323846f, 3.14159265358979323846f);
    // sin x ~ x (a0 + a1 x^2 + ... + a4 x^8), cos x ~ b0 + b1 x^2 + ... + b4 x^8
    // on |x| <= pi/2 (the near-minimax fit of phasor_poly.py)
    const f32x2 a0 = pack2(9.999999766e-01f, 9.999999766e-01f);
    const f32x2 a1 = pack2(-1.666664763e-01f, -1.666664763e-01f);
    const f32x2 a2 = pack2(8.332899816e-03f, 8.332899816e-03f);
    const f32x2 a3 = pack2(-1.980089730e-04f, -1.980089730e-04f);
    const f32x2 a4 = pack2(2.590487534e-06f, 2.590487534e-06f);
    const f32x2 b0 = pack2(9.999999535e-01f, 9.999999535e-01f);
    const f32x2 b1 = pack2(-4.999990535e-01f, -4.999990535e-01f);
    const f32x2 b2 = pack2(4.166358468e-02f, 4.166358468e-02f);
    const f32x2 b3 = pack2(-1.385370418e-03f, -1.385370418e-03f);
    const f32x2 b4 = pack2(2.315392824e-05f, 2.315392824e-05f);
    // Tier 0's MUFU pairs take the phase in radians straight from frequencies
    // scaled by 2 pi once per chunk (one multiply per exponential fewer); the
    // polynomial pairs and the reducing tiers keep turns.
    f32x2 rx[NP], ry[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const bool rad = TIER == 0 && j >= NPOLY;
        rx[j] = rad ? mul2(nx[j], kTwoPi) : nx[j];
        ry[j] = rad ? mul2(ny[j], kTwoPi) : ny[j];
    }
#pragma unroll 2
    for (int p = 0; p < len; ++p) {
        const float2 q = sp[p];
        const f32x2 qx = pack2(q.x, q.x), qy = pack2(q.y, q.y);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            f32x2 p2 = mul2(ry[j], qy);
            f32x2 f, t;
            if (TIER == 2) {
                // as encode_points: f_i = fl(nu_i d_i - rint(p_i)) with one FMA
                f32x2 p1 = mul2(rx[j], qx);
                f32x2 n1 = sub2(kM, add2(p1, kM)), n2 = sub2(kM, add2(p2, kM));
                f32x2 g = add2(fma2(rx[j], qx, n1), fma2(ry[j], qy, n2));
                f = sub2(g, sub2(add2(g, kM), kM));
            } else {
                // t = nu_x dx + nu_y dy with one rounding of the sum (FMA);
                // t - rint(t) is exact.  Error at most ulp(64)/2 + ulp(32)/2
                // = 2.9e-6 turns for |t| < 64 (3.6e-7 for |t| < 8).
                t = fma2(rx[j], qx, p2);
                if (TIER == 1 || j < NPOLY) f = sub2(t, sub2(add2(t, kM), kM));
            }
            f32x2 cr, si;
            if (j < NPOLY) {
                f32x2 x = mul2(f, kPi), x2 = mul2(x, x);
                f32x2 s = fma2(x2, a4, a3);
                s = fma2(x2, s, a2);
                s = fma2(x2, s, a1);
                s = fma2(x2, s, a0);
                s = mul2(s, x);
                f32x2 c = fma2(x2, b4, b3);
                c = fma2(x2, c, b2);
                c = fma2(x2, c, b1);
                c = fma2(x2, c, b0);
                cr = mul2(sub2(c, s), add2(c, s));  // cos 2x = (c - s)(c + s)
                si = mul2(add2(c, c), s);           // sin 2x = 2 c s
            } else {
                // tier 0: t is already in radians
                float2 a = unpack2(TIER == 0 ? t : mul2(f, kTwoPi));
                float s0, c0, s1, c1;
                __sincosf(a.x, &s0, &c0);
                __sincosf(a.y, &s1, &c1);
                cr = pack2(c0, c1);
                si = pack2(s0, s1);
            }
            ac[j] = add2(ac[j], cr);
            as[j] = add2(as[j], si);
        }
    }
}

// NPOLY < 0 selects the mixed form: warp w uses (w < poly_warps) + (w <
// poly_warps - 8) polynomial pairs, the others none, so the polynomial share is
// poly_warps / (8 NP) of the exponentials for poly_warps in 0 .. 16 (warps of an
// SM share its MUFU and FMA pipes).
// One (chunk, frequency slice) work item, executed by the whole CTA (256
// threads; contains __syncthreads).  sp and s_bound are the CTA's shared
// staging buffers; out receives the chunk's partial memory (or, with ATOMIC,
// is the map's memories).
template <int NP, int NPOLY, bool ATOMIC, bool FUSED>
__device__ __forceinline__ void encode_chunk_x2_body(const float2 *__restrict__ pts, int4 ch,
                                                     int c, int slice,
                                                     const float *__restrict__ nu, int D,
                                                     float nu_max_x, float nu_max_y,
                                                     int poly_warps, const PatchDev &pt,
                                                     float2 *__restrict__ out,
                                                     const TailSum &tail, float2 *sp,
                                                     unsigned *s_bound, int *s_tail)
{
    using namespace sm100;
    // a chunk holds at most kMaxChunk points (the staging buffer's size)
    const int len = VSAOGM_IN_BOUNDS(ch.z >= ch.y && ch.z - ch.y <= kMaxChunk) ? ch.z - ch.y : 0;
    const int kbase = slice * (512 * NP) + threadIdx.x;
    f32x2 nx[NP], ny[NP], ac[NP], as[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        int k0 = kbase + (2 * j) * 256, k1 = k0 + 256;
        nx[j] = pack2(k0 < D ? nu[k0] : 0.f, k1 < D ? nu[k1] : 0.f);
        ny[j] = pack2(k0 < D ? nu[D + k0] : 0.f, k1 < D ? nu[D + k1] : 0.f);
        ac[j] = pack2(0.f, 0.f);
        as[j] = pack2(0.f, 0.f);
    }
    if (threadIdx.x < 2) s_bound[threadIdx.x] = 0u;
    __syncthreads();
    float mx = 0.f, my = 0.f;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        float2 q = pts[ch.y + i];
        sp[i] = q;
        mx = fmaxf(mx, fabsf(q.x));
        my = fmaxf(my, fabsf(q.y));
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&s_bound[0], __float_as_uint(mx));
        atomicMax(&s_bound[1], __float_as_uint(my));
    }
    __syncthreads();
    const float ex = __uint_as_float(s_bound[0]) * nu_max_x;
    const float ey = __uint_as_float(s_bound[1]) * nu_max_y;
    const int tier = (ex < 4.0f && ey < 4.0f) ? 0 : (ex < 32.0f && ey < 32.0f) ? 1 : 2;
    if (NPOLY >= 0) {
        constexpr int P = NPOLY < 0 ? 0 : NPOLY;
        if (tier == 0)
            encode_points_x2<NP, P, 0>(sp, len, nx, ny, ac, as);
        else if (tier == 1)
            encode_points_x2<NP, P, 1>(sp, len, nx, ny, ac, as);
        else
            encode_points_x2<NP, P, 2>(sp, len, nx, ny, ac, as);
    } else if (tier == 2) {
        // the exact reduction leaves the FMA pipe no room for polynomial
        // exponentials: every warp takes the MUFU path
        encode_points_x2<NP, 0, 2>(sp, len, nx, ny, ac, as);
    } else if ((int)(threadIdx.x >> 5) < poly_warps - 8) {
        if (tier == 0)
            encode_points_x2<NP, 2, 0>(sp, len, nx, ny, ac, as);
        else
            encode_points_x2<NP, 2, 1>(sp, len, nx, ny, ac, as);
    } else if ((int)(threadIdx.x >> 5) < poly_warps) {
        if (tier == 0)
            encode_points_x2<NP, 1, 0>(sp, len, nx, ny, ac, as);
        else
            encode_points_x2<NP, 1, 1>(sp, len, nx, ny, ac, as);
    } else {
        if (tier == 0)
            encode_points_x2<NP, 0, 0>(sp, len, nx, ny, ac, as);
        else
            encode_points_x2<NP, 0, 1>(sp, len, nx, ny, ac, as);
    }
    const int mem = ch.x / pt.n, patch = ch.x - mem * pt.n;
    const float pcx = pt.n > 1 ? pt.cx[patch % pt.nx] : 0.f;
    const float pcy = pt.n > 1 ? pt.cy[patch / pt.nx] : 0.f;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const float2 cr = unpack2(ac[j]), si = unpack2(as[j]);
        // the frequencies again, from memory (registers held no turn-valued
        // copy of the MUFU pairs through the point loop)
        const int k0 = kbase + (2 * j) * 256, k1 = k0 + 256;
        const float2 vx = make_float2(k0 < D ? __ldg(nu + k0) : 0.f, k1 < D ? __ldg(nu + k1) : 0.f);
        const float2 vy = make_float2(k0 < D ? __ldg(nu + D + k0) : 0.f,
                                      k1 < D ? __ldg(nu + D + k1) : 0.f);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int k = kbase + (2 * j + h) * 256;
            float re = h ? cr.y : cr.x, im = h ? si.y : si.x;
            if (pt.n > 1) patch_rotate(h ? vx.y : vx.x, h ? vy.y : vy.x, pcx, pcy, re, im);
            if (k < D) {
                if (ATOMIC) {
                    float2 *w = out + (size_t)mem * D + k;
                    atomicAdd(&w->x, re);
                    atomicAdd(&w->y, im);
                } else {
                    out[(size_t)c * D + k] = make_float2(re, im);
                }
            }
        }
    }
    if (!ATOMIC && FUSED && tail.cnt) {
        // The bundling's sum (Eq. bundling) over this memory's chunks, fused:
        // every CTA publishes its partial and counts itself in; the last one
        // for this (memory, slice) adds the memory's partials for the slice in
        // chunk order (a fixed order, so the result does not depend on which
        // CTA is last) and clears the counter.
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            const int c0 = tail.cbeg[mem * pt.n], c1 = tail.cbeg[(mem + 1) * pt.n];
            unsigned *cnt = tail.cnt + (size_t)mem * tail.n_slices + slice;
            const bool last = atomicAdd(cnt, 1u) + 1u == (unsigned)(c1 - c0);
            if (last) *cnt = 0u;
            s_tail[0] = last ? 1 : 0;
            s_tail[1] = c0;
            s_tail[2] = c1;
        }
        __syncthreads();
        if (s_tail[0]) {
            __threadfence();
            const int c0 = s_tail[1], c1 = s_tail[2];
            float sr[2 * NP], si[2 * NP];
#pragma unroll
            for (int q = 0; q < 2 * NP; ++q) sr[q] = si[q] = 0.f;
            if (VSAOGM_IN_BOUNDS(c0 >= 0 && c1 >= c0))
                for (int cc = c0; cc < c1; ++cc) {
#pragma unroll
                    for (int q = 0; q < 2 * NP; ++q) {
                        const int k = kbase + q * 256;
                        if (k < D) {
                            const float2 v = __ldcg(out + (size_t)cc * D + k);
                            sr[q] += v.x;
                            si[q] += v.y;
                        }
                    }
                }
#pragma unroll
            for (int q = 0; q < 2 * NP; ++q) {
                const int k = kbase + q * 256;
                if (k < D) {
                    float2 *w = tail.omega + (size_t)mem * D + k;
                    const float2 o = *w;
                    *w = make_float2(o.x + sr[q], o.y + si[q]);
                }
            }
        }
    }
}

template <int NP, int NPOLY, bool ATOMIC, bool FUSED>
__global__ void __launch_bounds__(256, 4) encode_chunk_x2_kernel(const float2 *__restrict__ pts,
                                                              const int4 *__restrict__ chunks,
                                                              const int *__restrict__ n_chunks,
                                                              const float *__restrict__ nu, int D,
                                                              float nu_max_x, float nu_max_y,
                                                              int poly_warps, PatchDev pt,
                                                              float2 *__restrict__ out,
                                                              TailSum tail)
{
    __shared__ float2 sp[kMaxChunk];
    __shared__ unsigned s_bound[2];
    __shared__ int s_tail[3];
    const int nch = *n_chunks;
    if ((int)blockIdx.x >= nch) return;
    // the chunk of this launch position (longest first, see seg_meta_body)
    const int w = chunks[blockIdx.x].w;
    const int c = VSAOGM_IN_BOUNDS(w >= 0 && w < nch) ? w : (int)blockIdx.x;
    encode_chunk_x2_body<NP, NPOLY, ATOMIC, FUSED>(pts, chunks[c], c, blockIdx.y, nu, D,
                                                   nu_max_x, nu_max_y, poly_warps, pt, out, tail,
                                                   sp, s_bound, s_tail);
}

// 5''. Many maps in one persistent launch.  Work items are (map, chunk,
//      frequency slice), numbered map-major, chunk-major, slice-minor (the
//      slices of a chunk reuse its points from L2); each CTA takes the next
//      item from a global counter until none is left, so maps of any size and
//      dimension share the GPU evenly.
__global__ void __launch_bounds__(256) encode_batch_kernel(const __grid_constant__ BatchEncodeTable tab,
                                                           unsigned long long *counter)
{
    __shared__ float2 sp[kMaxChunk];
    __shared__ unsigned s_bound[2];
    __shared__ int s_tail[3];
    __shared__ long long s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long it = s_item;
        if (it >= tab.total) break;
        int lo = 0, hi = tab.n_maps - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (tab.m[mid].item_begin <= it) lo = mid; else hi = mid - 1;
        }
        const BatchEncodeMap &M = tab.m[lo];
        const long long local = it - M.item_begin;
        const int ci = (int)(local / M.slices), slice = (int)(local % M.slices);
        const int nch = *M.n_chunks;
        // the chunk of this position in the map's launch order (longest first)
        const int w = ci < nch ? M.chunks[ci].w : 0;
        const int c = VSAOGM_IN_BOUNDS(w >= 0 && w < nch) ? w : ci;
        if (ci < nch)
            encode_chunk_x2_body<4, -1, false, true>(M.pts, M.chunks[c], c, slice, M.nu, M.D,
                                                     M.nu_max_x, M.nu_max_y, M.poly_warps,
                                                     M.pt, M.out, M.tail, sp, s_bound, s_tail);
        __syncthreads();  // the staging buffers are reused by the next item
    }
}

// 6. omega[s][k] += the sum of the partial memories of memory s (the chunks
//    c0 .. c1 - 1 of its `patches` segments, which are contiguous), for the
//    kReduceFreqs frequencies k0 .. of one CTA, in a fixed order: warp w adds
//    chunks c0 + w, c0 + w + 8, ... (lane l frequency k0 + l), then warp 0
//    adds the eight warps' sums in warp order.  Spreading one memory's chunks
//    over eight warps keeps the heaviest memory from setting the time alone.
constexpr int kReduceFreqs = 32;
__device__ __forceinline__ void chunk_sum(const float2 *__restrict__ partial, int c0, int c1,
                                          int D, int k0, float2 *__restrict__ omega_row)
{
    __shared__ float2 part[8][kReduceFreqs];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, k = k0 + lane;
    float sr = 0.f, si = 0.f;
    if (k < D) {
#pragma unroll 4
        for (int c = c0 + warp; c < c1; c += 8) {
            const float2 v = partial[(size_t)c * D + k];
            sr += v.x;
            si += v.y;
        }
    }
    part[warp][lane] = make_float2(sr, si);
    __syncthreads();
    if (warp == 0 && k < D) {
        float tr = 0.f, ti = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            tr += part[w][lane].x;
            ti += part[w][lane].y;
        }
        const float2 o = omega_row[k];
        omega_row[k] = make_float2(o.x + tr, o.y + ti);
    }
}

// 6'. The fixed-order partial sums of many maps in one launch (maps whose
//     memories hold many chunks each): blockIdx.x is a global memory (maps'
//     memories numbered one after the other; beyond the 65535 limit of a
//     grid's y extent), blockIdx.y a range of kReduceFreqs frequencies.
__global__ void __launch_bounds__(256) reduce_batch_kernel(const __grid_constant__ BatchReduceTable tab)
{
    const int gs = blockIdx.x;
    int lo = 0, hi = tab.n_maps - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tab.m[mid].seg_begin <= gs) lo = mid; else hi = mid - 1;
    }
    const BatchReduceMap &M = tab.m[lo];
    const int s = gs - M.seg_begin;  // memory of this map; its patches' chunks are contiguous
    const int k0 = blockIdx.y * kReduceFreqs;
    if (k0 >= M.D) return;  // the whole CTA: the map's D ends before this range
    const int c0 = M.cbeg[s * M.patches], c1 = M.cbeg[(s + 1) * M.patches];
    if (c0 == c1 || !VSAOGM_IN_BOUNDS(c0 >= 0 && c1 > c0)) return;
    chunk_sum(M.partial, c0, c1, M.D, k0, M.omega + (size_t)s * M.D);
}

// 6. The same for one map: blockIdx.y is the memory, blockIdx.x a range of
//    kReduceFreqs frequencies.
__global__ void __launch_bounds__(256) reduce_partials_kernel(const float2 *__restrict__ partial,
                                                              const int *__restrict__ cbeg, int D,
                                                              int patches,
                                                              float2 *__restrict__ omega)
{
    const int s = blockIdx.y;
    const int k0 = blockIdx.x * kReduceFreqs;
    const int c0 = cbeg[s * patches], c1 = cbeg[(s + 1) * patches];
    if (c0 == c1 || !VSAOGM_IN_BOUNDS(c0 >= 0 && c1 > c0)) return;
    chunk_sum(partial, c0, c1, D, k0, omega + (size_t)s * D);
}

// Warps per CTA (of 8) that evaluate one frequency pair by polynomial when the
// map does not say otherwise: the share of exponentials moved from the MUFU
// pipe to the FMA pipe that balanced the two pipes on GB300 (measured sweeps).
// Chunks whose phases stay below 4 turns spend fewer FMA operations on the MUFU
// path, so more exponentials go to the polynomial there.
constexpr int kAutoPolyWarps4Near = 9;  // 4 pairs per thread, phases below 4 turns: 9/32
constexpr int kAutoPolyWarps4 = 6;      // 4 pairs per thread otherwise: 6/32
constexpr int kAutoPolyWarps2 = 3;      // 2 pairs per thread: 3/16

// cbeg non-null: the chunk sums run inside the launch (the last CTA of each
// memory and slice adds the memory's chunks in order; see encode_chunk_x2_body)
template <int NP, int NPOLY>
cudaError_t launch_x2(const vsaogm_map *m, const PatchDev &pt, const float2 *pts,
                      const int4 *chunks, const int *n_chunks, float2 *out, int max_chunks,
                      bool atomic, int pw, cudaStream_t st, const int *cbeg = nullptr)
{
    const int D = m->cfg.D;
    dim3 grid(max_chunks, (D + 512 * NP - 1) / (512 * NP));
    const TailSum tail{cbeg, m->enc_cnt, m->omega, (int)grid.y};
    if (atomic)
        encode_chunk_x2_kernel<NP, NPOLY, true, false><<<grid, 256, 0, st>>>(
            pts, chunks, n_chunks, m->nu, D, m->nu_max[0], m->nu_max[1], pw, pt, out, tail);
    else if (cbeg && NPOLY < 0)
        encode_chunk_x2_kernel<NP, NPOLY, false, NPOLY < 0><<<grid, 256, 0, st>>>(
            pts, chunks, n_chunks, m->nu, D, m->nu_max[0], m->nu_max[1], pw, pt, out, tail);
    else
        encode_chunk_x2_kernel<NP, NPOLY, false, false><<<grid, 256, 0, st>>>(
            pts, chunks, n_chunks, m->nu, D, m->nu_max[0], m->nu_max[1], pw, pt, out, tail);
    return cudaGetLastError();
}

// cbeg non-null asks for the fused chunk sums; returns in *fused whether the
// launch does them (the mixed-polynomial kernels only), else the caller sums.
cudaError_t launch_packed(const vsaogm_map *m, const PatchDev &pt, int np, const float2 *pts,
                          const int4 *chunks, const int *n_chunks, float2 *out, int max_chunks,
                          bool atomic, cudaStream_t st, const int *cbeg = nullptr,
                          bool *fused = nullptr)
{
    if (fused) *fused = false;
    const int npoly = std::min(m->encode_poly_pairs, np);
    const bool near = patches_near(m, pt);
    const int pw = m->encode_poly_warps >= 0
                       ? m->encode_poly_warps
                       : (np == 4 ? (near ? kAutoPolyWarps4Near : kAutoPolyWarps4) : kAutoPolyWarps2);
    if (npoly == 0 && pw > 0) {  // mixed: some warps with one polynomial pair
        if (fused) *fused = cbeg && !atomic;
        if (np == 4)
            return launch_x2<4, -1>(m, pt, pts, chunks, n_chunks, out, max_chunks, atomic, pw, st,
                                    cbeg);
        return launch_x2<2, -1>(m, pt, pts, chunks, n_chunks, out, max_chunks, atomic, pw, st,
                                cbeg);
    }
#define VSA_X2(NPV, NPOLYV) \
    launch_x2<NPV, NPOLYV>(m, pt, pts, chunks, n_chunks, out, max_chunks, atomic, 0, st)
    if (np == 4) {
        switch (npoly) {
            case 0: return VSA_X2(4, 0);
            case 1: return VSA_X2(4, 1);
            case 2: return VSA_X2(4, 2);
            default: return VSA_X2(4, 3);
        }
    }
    switch (npoly) {
        case 0: return VSA_X2(2, 0);
        case 1: return VSA_X2(2, 1);
        default: return VSA_X2(2, 2);
    }
#undef VSA_X2
}

template <int KPT>
cudaError_t launch_encode(const vsaogm_map *m, const PatchDev &pt, const float2 *pts,
                          const int4 *chunks, const int *n_chunks, float2 *out, int max_chunks,
                          bool atomic, cudaStream_t st)
{
    const int D = m->cfg.D;
    dim3 grid(max_chunks, (D + 256 * KPT - 1) / (256 * KPT));
    if (atomic)
        encode_chunk_kernel<KPT, true><<<grid, 256, 0, st>>>(
            pts, chunks, n_chunks, m->nu, D, m->nu_max[0], m->nu_max[1], pt, out);
    else
        encode_chunk_kernel<KPT, false><<<grid, 256, 0, st>>>(
            pts, chunks, n_chunks, m->nu, D, m->nu_max[0], m->nu_max[1], pt, out);
    return cudaGetLastError();
}

// The whole tile as its one patch (no rotation): the allocation-free path.
PatchDev single_patch()
{
    PatchDev p;
    p.n = p.nx = p.ny = 1;
    p.hw_x = p.hw_y = 0.f;
    p.inv_pw_x = p.inv_pw_y = 0.f;
    p.cx = p.cy = nullptr;
    return p;
}

}  // namespace

// Frequencies per thread and points per chunk for a batch of n points.
static void encode_shape(const vsaogm_map *m, int64_t n, int D, int *kpt, int *chunk)
{
    if (m->encode_packed)
        *kpt = D >= 4096 ? 8 : 4;
    else
        *kpt = D >= 4096 ? 4 : (D >= 2048 ? 2 : 1);
    int64_t slices = (D + 256 * *kpt - 1) / (256 * *kpt);
    int64_t target = 152 * 8 * 4;  // about four waves of 8 CTAs per SM
    int64_t c = std::max<int64_t>(1, n * slices / target);
    int p = 32;
    while (p * 2 <= c && p * 2 <= kMaxChunk) p *= 2;
    *chunk = p;
}

// Grows the encode scratch so that any batch of up to n points needs no
// allocation (the sizes encode_bundle asks for are monotone in n).
int reserve_encode(vsaogm_map *m, int64_t n64)
{
    const int n = (int)std::min<int64_t>(n64, kMaxBatch);
    if (n <= 0) return VSAOGM_OK;
    const int SP = m->S * std::max(m->patches[0].n, m->patches[1].n), S1 = SP + 1, D = m->cfg.D;
    int kpt, chunk;
    encode_shape(m, n, D, &kpt, &chunk);
    const int nb = (n + kSortBlock - 1) / kSortBlock;
    // The chunk size grows with the batch, so the chunk count ceil(n'/chunk(n'))
    // peaks just before each doubling of the chunk: evaluate it there and at n.
    int max_chunks = 0;
    auto chunks_at = [&](int np) {
        int k2, c2;
        encode_shape(m, np, D, &k2, &c2);
        return (np + c2 - 1) / c2;
    };
    max_chunks = chunks_at(n);
    int lo = 1;
    while (lo < n) {  // binary-search-free walk: step to the next size where the chunk changes
        int c_lo, k_lo;
        encode_shape(m, lo, D, &k_lo, &c_lo);
        int hi = lo;
        while (hi < n) {
            int c_hi, k_hi;
            encode_shape(m, std::min(n, hi * 2), D, &k_hi, &c_hi);
            if (c_hi != c_lo) break;
            hi = std::min(n, hi * 2);
        }
        // the largest n' in [hi, 2 hi) with the same chunk as lo
        int a = hi, b = std::min(n, 2 * hi);
        while (a < b) {
            int mid = a + (b - a + 1) / 2, c_mid, k_mid;
            encode_shape(m, mid, D, &k_mid, &c_mid);
            if (c_mid == c_lo) a = mid; else b = mid - 1;
        }
        max_chunks = std::max(max_chunks, chunks_at(a));
        if (a >= n) break;
        lo = a + 1;
    }
    max_chunks += SP;
    int rc;
    if ((rc = ensure(m->ws.blk_hist, sizeof(int) * (size_t)nb * S1))) return rc;
    if ((rc = ensure(m->ws.seg_meta, sizeof(int) * (size_t)(3 * S1 + 2)))) return rc;
    if ((rc = ensure(m->ws.chunks, sizeof(int4) * (size_t)max_chunks))) return rc;
    if ((rc = ensure(m->ws.sorted, sizeof(float2) * (size_t)n))) return rc;
    if (!(m->cfg.flags & VSAOGM_FLAG_ATOMIC) &&
        (rc = ensure(m->ws.partial, sizeof(float2) * (size_t)max_chunks * D)))
        return rc;
    return VSAOGM_OK;
}

// The sort of one map's call (steps 1-4): one CTA for a small call, else the
// four kernels.  hist needs nb x (S + 1) ints only for the latter.
static cudaError_t launch_sort(const float2 *xy, const uint8_t *lab, int n, const AxisDev &ax,
                               const AxisDev &ay, const PatchDev &pt, int S, int chunk, int *hist,
                               int *meta, int4 *chunks, unsigned long long *rejected,
                               float2 *sorted, cudaStream_t st, int *launches)
{
    const int S1 = S + 1;
    cudaError_t e;
    if (sort_small(n, S1)) {
        const size_t smem = sizeof(int) * kSmallSortWarps * S1;
        if ((e = cudaFuncSetAttribute(seg_sort_small_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        seg_sort_small_kernel<<<1, 32 * kSmallSortWarps, smem, st>>>(
            xy, lab, n, ax, ay, pt, S, chunk, meta, chunks, rejected, sorted);
        *launches = 1;
        return cudaGetLastError();
    }
    const int nb = (n + kSortBlock - 1) / kSortBlock;
    const size_t smem_count = sizeof(int) * S1;
    const size_t smem_scatter = sizeof(int) * kSortWarps * S1;
    // opt-in to more than 48 KB of dynamic shared memory (a per-device setting)
    if ((e = cudaFuncSetAttribute(seg_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_scatter)) != cudaSuccess)
        return e;
    seg_count_kernel<<<nb, 256, smem_count, st>>>(xy, lab, n, ax, ay, pt, S, hist);
    seg_scan_kernel<<<(S1 + kScanCols - 1) / kScanCols, 32 * kScanWarps, 0, st>>>(hist, nb, S1,
                                                                                 meta);
    seg_meta_kernel<<<1, kScanThreads, 0, st>>>(meta, S, chunk, chunks, rejected);
    seg_scatter_kernel<<<nb, 256, smem_scatter, st>>>(xy, lab, n, ax, ay, pt, S, hist, meta,
                                                      sorted);
    *launches = 4;
    return cudaGetLastError();
}

int batch_sort_entry(vsaogm_map *m, Scratch &ws, const PatchDev &pt, const float *xy,
                     const uint8_t *lab, int n, int chunk, BatchSortMap *e, int *max_chunks)
{
    const int S = m->S * pt.n, S1 = S + 1, D = m->cfg.D;
    const int nb = (n + kSortBlock - 1) / kSortBlock;
    *max_chunks = (n + chunk - 1) / chunk + S;
    int rc;
    if ((rc = ensure(ws.blk_hist, sizeof(int) * (size_t)nb * S1))) return rc;
    if ((rc = ensure(ws.seg_meta, sizeof(int) * (size_t)(3 * S1 + 2)))) return rc;
    if ((rc = ensure(ws.chunks, sizeof(int4) * (size_t)*max_chunks))) return rc;
    if ((rc = ensure(ws.sorted, sizeof(float2) * (size_t)n))) return rc;
    if ((rc = ensure(ws.partial, sizeof(float2) * (size_t)*max_chunks * D))) return rc;
    e->xy = (const float2 *)xy;
    e->lab = lab;
    e->n = n;
    e->S = S;
    e->chunk = chunk;
    e->ax = axis_x(m);
    e->ay = axis_y(m);
    e->pt = pt;
    e->hist = (int *)ws.blk_hist.ptr;
    e->meta = (int *)ws.seg_meta.ptr;
    e->chunks = (int4 *)ws.chunks.ptr;
    e->sorted = (float2 *)ws.sorted.ptr;
    e->rejected = m->rejected;
    e->nb = nb;
    return VSAOGM_OK;
}

int sort_scan_ctas(int S1) { return (S1 + kScanCols - 1) / kScanCols; }

bool sort_small(int n, int S1) { return n <= kSmallSortPoints && S1 <= kSmallSortSegs; }

int launch_sort_small_batch(const BatchSortTable &tab, int max_s1, cudaStream_t st)
{
    if (tab.n_maps <= 0) return VSAOGM_OK;
    const size_t smem = sizeof(int) * kSmallSortWarps * max_s1;
    cudaError_t e = cudaFuncSetAttribute(batch_seg_sort_small_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "batch sort: shared memory");
    batch_seg_sort_small_kernel<<<tab.n_maps, 32 * kSmallSortWarps, smem, st>>>(tab);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "batch sort");
    return VSAOGM_OK;
}

int launch_sort_batch(const BatchSortTable &tab, int blocks, int segs, int max_s1,
                      cudaStream_t st)
{
    if (tab.n_maps <= 0 || blocks <= 0) return VSAOGM_OK;
    const size_t smem_count = sizeof(int) * max_s1;
    const size_t smem_scatter = sizeof(int) * kSortWarps * max_s1;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(batch_seg_scatter_kernel,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_scatter)) != cudaSuccess)
        return cuda_error(e, "batch sort: shared memory");
    batch_seg_count_kernel<<<blocks, 256, smem_count, st>>>(tab);
    batch_seg_scan_kernel<<<segs, 32 * kScanWarps, 0, st>>>(tab);
    batch_seg_meta_kernel<<<tab.n_maps, kScanThreads, 0, st>>>(tab);
    batch_seg_scatter_kernel<<<blocks, 256, smem_scatter, st>>>(tab);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "batch sort");
    return VSAOGM_OK;
}

const PatchDev &choose_patches(const vsaogm_map *m, int64_t n, int min_per_segment)
{
    const PatchDev &fine = m->patches[1], &coarse = m->patches[0];
    if (fine.n == coarse.n) return coarse;
    return n >= (int64_t)min_per_segment * m->S * fine.n ? fine : coarse;
}

bool patches_near(const vsaogm_map *m, const PatchDev &pt)
{
    return m->tile_w / (2.0 * pt.nx) * m->nu_max[0] < 4.0 &&
           m->tile_h / (2.0 * pt.ny) * m->nu_max[1] < 4.0;
}

void batch_encode_entry(const vsaogm_map *m, const Scratch &ws, const PatchDev &pt,
                        BatchEncodeMap *e)
{
    const int S1 = m->S * pt.n + 1;
    const int *meta = (const int *)ws.seg_meta.ptr;
    e->pts = (const float2 *)ws.sorted.ptr;
    e->chunks = (const int4 *)ws.chunks.ptr;
    e->n_chunks = meta + 3 * S1 + 1;
    e->nu = m->nu;
    e->out = (float2 *)ws.partial.ptr;
    e->D = m->cfg.D;
    e->slices = (m->cfg.D + 2047) / 2048;  // the batched kernel holds 8 frequencies a thread
    e->nu_max_x = m->nu_max[0];
    e->nu_max_y = m->nu_max[1];
    e->pt = pt;
    e->tail = TailSum{meta + 2 * S1 + 1, m->enc_cnt, m->omega, e->slices};
}

void batch_reduce_entry(const vsaogm_map *m, const Scratch &ws, const PatchDev &pt,
                        BatchReduceMap *e)
{
    const int S1 = m->S * pt.n + 1;
    const int *meta = (const int *)ws.seg_meta.ptr;
    e->partial = (const float2 *)ws.partial.ptr;
    e->cbeg = meta + 2 * S1 + 1;
    e->omega = m->omega;
    e->D = m->cfg.D;
    e->patches = pt.n;
}

int launch_reduce_batch(const BatchReduceTable &tab, int d_max, cudaStream_t st)
{
    reduce_batch_kernel<<<dim3(tab.total_segs, (d_max + kReduceFreqs - 1) / kReduceFreqs), 256, 0,
                          st>>>(tab);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VSAOGM_OK : cuda_error(e, "batch reduce");
}

int encode_batch_ctas()
{
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, encode_batch_kernel, 256, 0) !=
        cudaSuccess)
        per_sm = 1;
    return std::max(1, per_sm) * std::max(1, sms);
}

int launch_encode_batch(const BatchEncodeTable &tab, unsigned long long *counter, int ctas,
                        cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_error(e, "batch encode");
    encode_batch_kernel<<<ctas, 256, 0, st>>>(tab, counter);
    e = cudaGetLastError();
    return e == cudaSuccess ? VSAOGM_OK : cuda_error(e, "batch encode");
}

int encode_bundle(vsaogm_map *m, const float *xy_f, const uint8_t *lab, int64_t n64,
                  cudaStream_t st)
{
    const int n = (int)n64;
    const PatchDev &pt = choose_patches(m, n64);
    const int S = m->S * pt.n, S1 = S + 1, D = m->cfg.D;
    const bool atomic = (m->cfg.flags & VSAOGM_FLAG_ATOMIC) != 0;
    int kpt, chunk;
    encode_shape(m, n, D, &kpt, &chunk);
    const int nb = (n + kSortBlock - 1) / kSortBlock;
    const int max_chunks = (n + chunk - 1) / chunk + S;
    int rc;
    if ((rc = ensure(m->ws.blk_hist, sizeof(int) * (size_t)nb * S1))) return rc;
    if ((rc = ensure(m->ws.seg_meta, sizeof(int) * (size_t)(3 * S1 + 2)))) return rc;
    if ((rc = ensure(m->ws.chunks, sizeof(int4) * (size_t)max_chunks))) return rc;
    if ((rc = ensure(m->ws.sorted, sizeof(float2) * (size_t)n))) return rc;
    if (!atomic && (rc = ensure(m->ws.partial, sizeof(float2) * (size_t)max_chunks * D))) return rc;
    int *hist = (int *)m->ws.blk_hist.ptr, *meta = (int *)m->ws.seg_meta.ptr;
    int4 *chunks = (int4 *)m->ws.chunks.ptr;
    float2 *sorted = (float2 *)m->ws.sorted.ptr;
    const float2 *xy = (const float2 *)xy_f;
    AxisDev ax = axis_x(m), ay = axis_y(m);
    cudaError_t e;

    {
        StageScope sc(m, VSAOGM_STAGE_SORT, st);
        int launches = 0;
        if ((e = launch_sort(xy, lab, n, ax, ay, pt, S, chunk, hist, meta, chunks, m->rejected,
                             sorted, st, &launches)) != cudaSuccess)
            return cuda_error(e, "encode: sort");
        sc.end(launches);
    }
    const int *cbeg = meta + S1 + S1 + 1;
    const int *n_chunks = cbeg + S + 1;
    float2 *out = atomic ? m->omega : (float2 *)m->ws.partial.ptr;
    bool fused = false;
    {
        StageScope sc(m, VSAOGM_STAGE_ENCODE, st);
        // a call whose memories hold few chunks each sums them in the same
        // launch (one launch less on small calls); many chunks per memory keep
        // the separate reduction, which spreads each memory over many CTAs
        const bool want_fused = (n + chunk - 1) / chunk <= kFusedChunksPerMemory * m->S;
        if (m->encode_packed)
            e = launch_packed(m, pt, kpt / 2, sorted, chunks, n_chunks, out, max_chunks, atomic,
                              st, want_fused ? cbeg : nullptr, &fused);
        else if (kpt == 4)
            e = launch_encode<4>(m, pt, sorted, chunks, n_chunks, out, max_chunks, atomic, st);
        else if (kpt == 2)
            e = launch_encode<2>(m, pt, sorted, chunks, n_chunks, out, max_chunks, atomic, st);
        else
            e = launch_encode<1>(m, pt, sorted, chunks, n_chunks, out, max_chunks, atomic, st);
        if (e != cudaSuccess) return cuda_error(e, "encode: bundle");
        sc.end(1);
    }
    if (!atomic && !fused) {
        StageScope sc(m, VSAOGM_STAGE_REDUCE, st);
        dim3 grid((D + kReduceFreqs - 1) / kReduceFreqs, m->S);
        reduce_partials_kernel<<<grid, 256, 0, st>>>((const float2 *)m->ws.partial.ptr, cbeg, D,
                                                     pt.n, m->omega);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "encode: reduce");
        sc.end(1);
    }
    return VSAOGM_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free encode + bundle (vsaogm_encode_bundle_noalloc).
// ---------------------------------------------------------------------------
constexpr int kNoAllocMaxPoints = 1 << 18;
constexpr int kNoAllocMaxDevices = 64;

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (with that device current) and cached.  vsaogm_create calls this
// for its device, so the lookup (which under lazy module loading also loads
// this file's module and reserves the array) happens at set-up time and not
// in the first allocation-free call.
int noalloc_scratch(int device, unsigned char **out)
{
    static std::mutex mu;
    static unsigned char *addr[kNoAllocMaxDevices] = {};
    if (device < 0 || device >= kNoAllocMaxDevices)
        return set_error(VSAOGM_E_INVAL, "device %d out of range for the static scratch", device);
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "encode_noalloc: scratch address");
        addr[device] = (unsigned char *)p;
    }
    *out = addr[device];
    return VSAOGM_OK;
}

static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

static int encode_bundle_noalloc(vsaogm_map *m, const float *xy_f, const uint8_t *lab, int n,
                                 cudaStream_t st)
{
    // one patch per tile: the scratch bound below stays the one of the memories
    const PatchDev pt = single_patch();
    const int S = m->S, S1 = S + 1, D = m->cfg.D;
    int kpt, chunk;
    encode_shape(m, n, D, &kpt, &chunk);
    const int nb = (n + kSortBlock - 1) / kSortBlock;
    const int max_chunks = (n + chunk - 1) / chunk + S;
    const size_t b_hist = align256(sizeof(int) * (size_t)nb * S1);
    const size_t b_meta = align256(sizeof(int) * (size_t)(3 * S1 + 2));
    const size_t b_chunks = align256(sizeof(int4) * (size_t)max_chunks);
    const size_t b_sorted = align256(sizeof(float2) * (size_t)n);
    if (b_hist + b_meta + b_chunks + b_sorted > kNoAllocScratchBytes)
        return set_error(VSAOGM_E_INVAL,
                         "encode_noalloc: %d points need %zu bytes of scratch, more than the "
                         "static %zu",
                         n, b_hist + b_meta + b_chunks + b_sorted, kNoAllocScratchBytes);
    int device = -1;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_error(e, "encode_noalloc");
    if (device != m->device)
        return set_error(VSAOGM_E_INVAL, "encode_noalloc: the map's device is not current");
    unsigned char *base = nullptr;
    int rc = noalloc_scratch(device, &base);
    if (rc) return rc;
    int *hist = (int *)base;
    int *meta = (int *)(base + b_hist);
    int4 *chunks = (int4 *)(base + b_hist + b_meta);
    float2 *sorted = (float2 *)(base + b_hist + b_meta + b_chunks);
    const float2 *xy = (const float2 *)xy_f;
    AxisDev ax = axis_x(m), ay = axis_y(m);
    // Every scratch word these kernels read is written earlier in the same call
    // (histograms, offsets, chunk table, sorted points), so nothing has to be
    // cleared; bundling adds straight into the map's memories with atomics.
    int launches = 0;
    if ((e = launch_sort(xy, lab, n, ax, ay, pt, S, chunk, hist, meta, chunks, m->rejected,
                         sorted, st, &launches)) != cudaSuccess)
        return cuda_error(e, "encode_noalloc: sort");
    const int *n_chunks = meta + S1 + S1 + 1 + S + 1;
    if (m->encode_packed)
        e = launch_packed(m, pt, kpt / 2, sorted, chunks, n_chunks, m->omega, max_chunks, true,
                          st);
    else if (kpt == 4)
        e = launch_encode<4>(m, pt, sorted, chunks, n_chunks, m->omega, max_chunks, true, st);
    else if (kpt == 2)
        e = launch_encode<2>(m, pt, sorted, chunks, n_chunks, m->omega, max_chunks, true, st);
    else
        e = launch_encode<1>(m, pt, sorted, chunks, n_chunks, m->omega, max_chunks, true, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "encode_noalloc");
    return VSAOGM_OK;
}

VSAOGM_CHECK_TU(encode)

}  // namespace vsaogm_impl

extern "C" int vsaogm_encode_bundle_noalloc(vsaogm_map *m, const float *xy, const uint8_t *lab,
                                            int64_t n, void *stream)
{
    using namespace vsaogm_impl;
    if (!m) return set_error(VSAOGM_E_INVAL, "map is NULL");
    if (n < 0) return set_error(VSAOGM_E_INVAL, "n must be >= 0");
    if (n == 0) return VSAOGM_OK;
    ++m->mem_gen;
    if (n > kNoAllocMaxPoints)
        return set_error(VSAOGM_E_INVAL, "encode_noalloc: n = %lld exceeds the maximum of %d points",
                         (long long)n, kNoAllocMaxPoints);
    if (!xy || !lab) return set_error(VSAOGM_E_INVAL, "xy and labels must not be NULL");
    if ((uintptr_t)xy % 8 != 0) return set_error(VSAOGM_E_INVAL, "xy must be 8-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    // checked maps report rejected points as vsaogm_encode_bundle does: the
    // counter is read into host stack variables before and after (no allocation)
    const bool checked = (m->cfg.flags & VSAOGM_FLAG_CHECKED) != 0;
    unsigned long long before = 0, after = 0;
    cudaError_t e;
    if (checked && (e = cudaMemcpyAsync(&before, m->rejected, sizeof(before),
                                        cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_error(e, "encode_noalloc");
    int rc = encode_bundle_noalloc(m, xy, lab, (int)n, st);
    if (rc || !checked) return rc;
    if ((e = cudaMemcpyAsync(&after, m->rejected, sizeof(after), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_error(e, "encode_noalloc");
    if (after != before)
        return set_error(VSAOGM_E_DATA, "%llu points rejected (label > 1 or non-finite)",
                         after - before);
    return VSAOGM_OK;
}
