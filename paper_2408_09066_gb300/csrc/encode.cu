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
//                     tile-centred frame (offsets computed in FP64 per point).
//   5. encode_chunk : one CTA per (chunk, slice of k); each thread keeps KPT
//                     frequencies in registers, walks the chunk's points from
//                     shared memory and accumulates exp(i 2 pi nu . p) with
//                     MUFU sin/cos after an exact reduction of the phase to
//                     [-1/2, 1/2] turns.  Partial memories go to scratch ...
//   6. reduce       : ... and are summed per segment in a fixed order, so the
//                     result does not depend on scheduling.  With
//                     VSAOGM_FLAG_ATOMIC step 5 adds into the memories with
//                     atomics instead and step 6 is skipped.
#include <algorithm>

#include "internal.cuh"

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

// Segment 2 beta + psi, or S for a point that is rejected.
__device__ __forceinline__ int point_segment(float x, float y, unsigned lab, const AxisDev &ax,
                                             const AxisDev &ay, int S)
{
    if (lab > 1u || !isfinite(x) || !isfinite(y)) return S;
    int bx = tile_along(ax.bnd_lo, ax.n_tiles - 1, x);
    int by = tile_along(ay.bnd_lo, ay.n_tiles - 1, y);
    return 2 * (by * ax.n_tiles + bx) + (int)lab;
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

// 1. Per-block histogram over segments 0..S (S = rejected).
__global__ void __launch_bounds__(256) seg_count_kernel(const float2 *__restrict__ xy,
                                                        const uint8_t *__restrict__ lab, int n,
                                                        AxisDev ax, AxisDev ay, int S,
                                                        int *__restrict__ hist)
{
    extern __shared__ int cnt[];  // [S + 1]
    const int S1 = S + 1;
    for (int s = threadIdx.x; s < S1; s += blockDim.x) cnt[s] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = blockIdx.x * kSortBlock + warp * (kSortBlock / kSortWarps);
    for (int r = 0; r < kSortBlock / kSortWarps / 32; ++r) {
        int i = base + r * 32 + lane;
        int seg = -1;
        if (i < n) {
            float2 p = xy[i];
            seg = point_segment(p.x, p.y, lab[i], ax, ay, S);
        }
        unsigned peers = __match_any_sync(0xffffffffu, seg);
        if (seg >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[seg], __popc(peers));
    }
    __syncthreads();
    for (int s = threadIdx.x; s < S1; s += blockDim.x) hist[(size_t)blockIdx.x * S1 + s] = cnt[s];
}

// 2. Column s of hist [nb][S1] -> exclusive prefix over blocks (in place);
//    total[s] = column sum.
__global__ void __launch_bounds__(kScanThreads) seg_scan_kernel(int *__restrict__ hist, int nb,
                                                                int S1, int *__restrict__ total)
{
    const int s = blockIdx.x;
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += kScanThreads) {
        int b = b0 + threadIdx.x;
        int v = b < nb ? hist[(size_t)b * S1 + s] : 0;
        int tot;
        int pre = block_exclusive_scan(v, &tot);
        if (b < nb) hist[(size_t)b * S1 + s] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) total[s] = carry;
}

// 3. Segment bases, chunk table, rejected count.  One CTA.
//    meta layout: total[S1] | base[S1 + 1] | chunk_begin[S + 1] | n_chunks[1]
__global__ void __launch_bounds__(kScanThreads) seg_meta_kernel(int *__restrict__ meta, int S,
                                                                int chunk,
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
}

// 4. Stable scatter into segment order, tile-centred coordinates.
__global__ void __launch_bounds__(256) seg_scatter_kernel(const float2 *__restrict__ xy,
                                                          const uint8_t *__restrict__ lab, int n,
                                                          AxisDev ax, AxisDev ay, int S,
                                                          const int *__restrict__ blk_off,
                                                          const int *__restrict__ meta,
                                                          float2 *__restrict__ sorted)
{
    extern __shared__ int wcnt[];  // [kSortWarps][S1]: counts, then running cursors
    const int S1 = S + 1;
    const int *seg_base = meta + S1;
    for (int s = threadIdx.x; s < kSortWarps * S1; s += blockDim.x) wcnt[s] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = blockIdx.x * kSortBlock + warp * (kSortBlock / kSortWarps);
    const int rounds = kSortBlock / kSortWarps / 32;
    int *mine = wcnt + warp * S1;
    // pass 1: per-warp counts (only this warp touches its row)
    for (int r = 0; r < rounds; ++r) {
        int i = base + r * 32 + lane;
        int seg = -1;
        if (i < n) {
            float2 p = xy[i];
            seg = point_segment(p.x, p.y, lab[i], ax, ay, S);
        }
        unsigned peers = __match_any_sync(0xffffffffu, seg);
        if (seg >= 0 && lane == __ffs(peers) - 1) mine[seg] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // cursors: global position of each warp's first point of each segment
    for (int s = threadIdx.x; s < S1; s += blockDim.x) {
        int run = seg_base[s] + blk_off[(size_t)blockIdx.x * S1 + s];
        for (int w = 0; w < kSortWarps; ++w) {
            int c = wcnt[w * S1 + s];
            wcnt[w * S1 + s] = run;
            run += c;
        }
    }
    __syncthreads();
    // pass 2: ranks in original order, write tile-centred coordinates
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < rounds; ++r) {
        int i = base + r * 32 + lane;
        int seg = -1;
        float2 p = make_float2(0.f, 0.f);
        if (i < n) {
            p = xy[i];
            seg = point_segment(p.x, p.y, lab[i], ax, ay, S);
        }
        unsigned peers = __match_any_sync(0xffffffffu, seg);
        int dst = 0;
        if (seg >= 0) dst = mine[seg] + __popc(peers & lt);
        __syncwarp();
        if (seg >= 0 && lane == __ffs(peers) - 1) mine[seg] += __popc(peers);
        __syncwarp();
        if (seg >= 0 && seg < S) {
            int beta = seg >> 1;
            int bx = beta % ax.n_tiles, by = beta / ax.n_tiles;
            // FP64 once per point: the offset from the tile centre, then f32.
            float dx = (float)((double)p.x - ax.centre[bx]);
            float dy = (float)((double)p.y - ay.centre[by]);
            sorted[dst] = make_float2(dx, dy);
        }
    }
}

// 5. Encode + bundle one chunk of one segment over a slice of 256*KPT
//    frequencies.  The phase in turns t = nu_x dx + nu_y dy is reduced to
//    f = t - rint(t) in [-1/2, 1/2] and then one MUFU sin and one MUFU cos of
//    2 pi f are taken.
//    Fast reduction (every |nu dx|, |nu dy| of the chunk below 32 turns):
//      p1 = fl(nu_x dx), p2 = fl(nu_y dy), r = rint(p1 + p2),
//      f = fl(fl(p1 - r) + p2); p1 - r is exact (both are multiples of
//      ulp(p1) and |p1 - r| <= |p2| + 1/2), so the only phase errors are the
//      two product roundings, at most ulp(32)/2 = 2^-19 turns each.
//    Exact reduction (points far from their tile centre, e.g. outside the
//      map): the product errors e1, e2 are recovered with FMA (TwoProduct)
//      and added after the reduction, leaving an error of about 2^-24 turns.
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
            float r = __fsub_rn(__fadd_rn(__fadd_rn(p1, p2), kMagic), kMagic);
            float f = __fadd_rn(__fsub_rn(p1, r), p2);
            if (EXACT) {
                float e1 = fmaf(nx[j], q.x, -p1);
                float e2 = fmaf(ny[j], q.y, -p2);
                f = __fadd_rn(f, __fadd_rn(e1, e2));
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
                                                           float2 *__restrict__ out)
{
    __shared__ float2 sp[kMaxChunk];
    __shared__ unsigned s_bound[2];
    const int c = blockIdx.x;
    if (c >= *n_chunks) return;
    const int4 ch = chunks[c];
    const int len = ch.z - ch.y;
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
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        int k = kbase + j * 256;
        if (k < D) {
            if (ATOMIC) {
                float2 *w = out + (size_t)ch.x * D + k;
                atomicAdd(&w->x, ar[j]);
                atomicAdd(&w->y, ai[j]);
            } else {
                out[(size_t)c * D + k] = make_float2(ar[j], ai[j]);
            }
        }
    }
}

// 6. omega[s][k] += sum of the partial memories of segment s, in chunk order.
__global__ void __launch_bounds__(256) reduce_partials_kernel(const float2 *__restrict__ partial,
                                                              const int *__restrict__ cbeg, int D,
                                                              float2 *__restrict__ omega)
{
    const int s = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= D) return;
    const int c0 = cbeg[s], c1 = cbeg[s + 1];
    if (c0 == c1) return;
    float sr = 0.f, si = 0.f;
    for (int c = c0; c < c1; ++c) {
        float2 v = partial[(size_t)c * D + k];
        sr += v.x;
        si += v.y;
    }
    float2 w = omega[(size_t)s * D + k];
    omega[(size_t)s * D + k] = make_float2(w.x + sr, w.y + si);
}

template <int KPT>
cudaError_t launch_encode(const vsaogm_map *m, const float2 *pts, const int4 *chunks,
                          const int *n_chunks, float2 *out, int max_chunks, bool atomic,
                          cudaStream_t st)
{
    const int D = m->cfg.D;
    dim3 grid(max_chunks, (D + 256 * KPT - 1) / (256 * KPT));
    if (atomic)
        encode_chunk_kernel<KPT, true><<<grid, 256, 0, st>>>(pts, chunks, n_chunks, m->nu, D,
                                                             m->nu_max[0], m->nu_max[1], out);
    else
        encode_chunk_kernel<KPT, false><<<grid, 256, 0, st>>>(pts, chunks, n_chunks, m->nu, D,
                                                              m->nu_max[0], m->nu_max[1], out);
    return cudaGetLastError();
}

}  // namespace

// Frequencies per thread and points per chunk for a batch of n points.
static void encode_shape(int64_t n, int D, int *kpt, int *chunk)
{
    *kpt = D >= 4096 ? 4 : (D >= 2048 ? 2 : 1);
    int64_t slices = (D + 256 * *kpt - 1) / (256 * *kpt);
    int64_t target = 152 * 8 * 4;  // about four waves of 8 CTAs per SM
    int64_t c = std::max<int64_t>(1, n * slices / target);
    int p = 32;
    while (p * 2 <= c && p * 2 <= kMaxChunk) p *= 2;
    *chunk = p;
}

int encode_bundle(vsaogm_map *m, const float *xy_f, const uint8_t *lab, int64_t n64,
                  cudaStream_t st)
{
    const int n = (int)n64;
    const int S = m->S, S1 = S + 1, D = m->cfg.D;
    const bool atomic = (m->cfg.flags & VSAOGM_FLAG_ATOMIC) != 0;
    int kpt, chunk;
    encode_shape(n, D, &kpt, &chunk);
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

    size_t smem_count = sizeof(int) * S1;
    size_t smem_scatter = sizeof(int) * kSortWarps * S1;
    // opt-in to more than 48 KB of dynamic shared memory (a per-device setting)
    if ((e = cudaFuncSetAttribute(seg_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_scatter)) != cudaSuccess)
        return cuda_error(e, "encode: shared memory");
    {
        StageScope sc(m, VSAOGM_STAGE_SORT, st);
        seg_count_kernel<<<nb, 256, smem_count, st>>>(xy, lab, n, ax, ay, S, hist);
        seg_scan_kernel<<<S1, kScanThreads, 0, st>>>(hist, nb, S1, meta);
        seg_meta_kernel<<<1, kScanThreads, 0, st>>>(meta, S, chunk, chunks, m->rejected);
        seg_scatter_kernel<<<nb, 256, smem_scatter, st>>>(xy, lab, n, ax, ay, S, hist, meta,
                                                          sorted);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "encode: sort");
        sc.end(4);
    }
    const int *cbeg = meta + S1 + S1 + 1;
    const int *n_chunks = cbeg + S + 1;
    float2 *out = atomic ? m->omega : (float2 *)m->ws.partial.ptr;
    {
        StageScope sc(m, VSAOGM_STAGE_ENCODE, st);
        if (kpt == 4)
            e = launch_encode<4>(m, sorted, chunks, n_chunks, out, max_chunks, atomic, st);
        else if (kpt == 2)
            e = launch_encode<2>(m, sorted, chunks, n_chunks, out, max_chunks, atomic, st);
        else
            e = launch_encode<1>(m, sorted, chunks, n_chunks, out, max_chunks, atomic, st);
        if (e != cudaSuccess) return cuda_error(e, "encode: bundle");
        sc.end(1);
    }
    if (!atomic) {
        StageScope sc(m, VSAOGM_STAGE_REDUCE, st);
        dim3 grid((D + 255) / 256, S);
        reduce_partials_kernel<<<grid, 256, 0, st>>>((const float2 *)m->ws.partial.ptr, cbeg, D,
                                                     m->omega);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "encode: reduce");
        sc.end(1);
    }
    return VSAOGM_OK;
}

}  // namespace vsaogm_impl
