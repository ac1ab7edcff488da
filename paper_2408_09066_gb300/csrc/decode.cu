// Decoding (Eqs. vector-normalization, loc-query, non-linearities).
//
// For a cell (i, j) in tile beta and class psi,
//   P = Re sum_k conj(w_k) A[i,k] B[j,k] / ||w||,
//   A[i,k] = exp(i 2 pi nu_x[k] dx_i), B[j,k] = exp(i 2 pi nu_y[k] dy_j),
// with w the memory 2 beta + psi and (dx_i, dy_j) the cell centre relative to
// the tile centre (the frame the memories are kept in).  This is the
// separable form of Eq. loc-query: the location vector of a cell factors into
// an x part shared by a column and a y part shared by a row.
//
// The FP32 path below is a SIMT contraction that builds A and
// U_psi = conj(w_hat_psi) * B in shared memory (sin/cos on the fly, never read
// from HBM) and accumulates both classes of a 64 x 64 block of cells per CTA.
// The per-class maximum over the map is folded into the epilogue with an
// order-preserving atomicMax.
#include <algorithm>

#include "internal.cuh"

namespace vsaogm_impl {
namespace {

constexpr int kBI = 64, kBJ = 64, kKC = 32;  // cells per block (x, y), k per stage

// ||w|| per memory -> 1/||w|| (0 for an all-zero memory).
// ||w_s||^2 by one CTA of kNormThreads threads: each thread keeps four running
// sums (frequencies k = t + j kNormThreads, j mod 4) so that four loads are in
// flight, then a fixed-order tree over the warps (the same order on every call).
constexpr int kNormThreads = 1024;

__device__ __forceinline__ float norm2_row(const float2 *__restrict__ w, int D)
{
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    int k = threadIdx.x;
    for (; k + 3 * kNormThreads < D; k += 4 * kNormThreads) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 v = w[k + j * kNormThreads];
            a[j] = fmaf(v.x, v.x, fmaf(v.y, v.y, a[j]));
        }
    }
    for (int j = 0; k < D; k += kNormThreads, ++j) {
        const float2 v = w[k];
        a[j & 3] = fmaf(v.x, v.x, fmaf(v.y, v.y, a[j & 3]));
    }
    float acc = (a[0] + a[1]) + (a[2] + a[3]);
    __shared__ float red[kNormThreads / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x < 32) {
        t = red[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

__global__ void __launch_bounds__(kNormThreads) norms_kernel(const float2 *__restrict__ omega,
                                                             int D, float *__restrict__ inv_norm)
{
    const int s = blockIdx.x;
    const float t = norm2_row(omega + (size_t)s * D, D);
    if (threadIdx.x == 0) inv_norm[s] = t > 0.f ? rsqrtf(t) : 0.f;
}

// exp(i 2 pi nu d) with the phase reduced exactly to [-1/2, 1/2] turns:
// p + e = nu * d exactly (FMA), r = rint(p), f = (p - r) + e.
__device__ __forceinline__ float2 unit_phasor(float nu, float d)
{
    const float kMagic = 12582912.0f;
    float p = __fmul_rn(nu, d);
    float e = fmaf(nu, d, -p);
    float r = __fsub_rn(__fadd_rn(p, kMagic), kMagic);
    float f = __fadd_rn(__fsub_rn(p, r), e);
    float s, c;
    __sincosf(__fmul_rn(f, 6.28318530717958647692f), &s, &c);
    return make_float2(c, s);
}

// One block of cells over one slice [k_begin, k_end) of the frequencies; the
// partial maps of the slices are summed by reduce_slices_kernel.
__global__ void __launch_bounds__(256) decode_fp32_kernel(
    const BlockBatch blocks, const float2 *__restrict__ omega, const float *__restrict__ inv_norm,
    const float *__restrict__ nu, int D, OutGeom og, const float *__restrict__ col_off,
    const float *__restrict__ row_off, int k_per_split, float *__restrict__ partial)
{
    __shared__ float2 sA[kKC][kBI];
    __shared__ float2 sU[2][kKC][kBJ];
    const DecodeBlock b = blocks.b[blockIdx.x];
    const int split = blockIdx.y;
    const int k_first = split * k_per_split;
    const int k_last = min(D, k_first + k_per_split);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const float w0 = inv_norm[2 * b.tile], w1 = inv_norm[2 * b.tile + 1];
    const float2 *om0 = omega + (size_t)(2 * b.tile) * D;
    const float2 *om1 = om0 + D;
    float acc[2][4][4];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[c][u][v] = 0.f;

    for (int k0 = k_first; k0 < k_last; k0 += kKC) {
        // tables for this stage: 2048 A entries and 2048 B entries (x2 classes)
        for (int e = threadIdx.x; e < kKC * kBI; e += blockDim.x) {
            int kk = e / kBI, ii = e % kBI;
            int k = k0 + kk, i = b.i0 + ii;
            float2 a = make_float2(0.f, 0.f);
            if (k < k_last && i < b.i1) a = unit_phasor(nu[k], col_off[i]);
            sA[kk][ii] = a;
        }
        for (int e = threadIdx.x; e < kKC * kBJ; e += blockDim.x) {
            int kk = e / kBJ, jj = e % kBJ;
            int k = k0 + kk, j = b.j0 + jj;
            float2 u0 = make_float2(0.f, 0.f), u1 = u0;
            if (k < k_last && j < b.j1) {
                float2 bb = unit_phasor(nu[D + k], row_off[j]);
                float2 m0 = om0[k], m1 = om1[k];
                // conj(w_hat) * B
                u0 = make_float2(w0 * (m0.x * bb.x + m0.y * bb.y), w0 * (m0.x * bb.y - m0.y * bb.x));
                u1 = make_float2(w1 * (m1.x * bb.x + m1.y * bb.y), w1 * (m1.x * bb.y - m1.y * bb.x));
            }
            sU[0][kk][jj] = u0;
            sU[1][kk][jj] = u1;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kKC; ++kk) {
            float2 a[4], u[2][4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = sA[kk][tx + 16 * q];
                u[0][q] = sU[0][kk][ty + 16 * q];
                u[1][q] = sU[1][kk][ty + 16 * q];
            }
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int v = 0; v < 4; ++v)
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        acc[c][v][q] = fmaf(u[c][v].x, a[q].x, fmaf(-u[c][v].y, a[q].y, acc[c][v][q]));
        }
        __syncthreads();
    }
    // epilogue: this slice's partial maps
    float *out = partial + (size_t)split * 2 * og.OH * og.OW;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        int j = b.j0 + ty + 16 * v;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int i = b.i0 + tx + 16 * q;
            if (i < b.i1 && j < b.j1) {
#pragma unroll
                for (int c = 0; c < 2; ++c)
                    out[((size_t)c * og.OH + (j - og.oy)) * og.OW + (i - og.ox)] = acc[c][v][q];
            }
        }
    }
}

// heat = (sum of the slices' partial maps, in slice order) * inv_scale, and
// the per-class maxima of Eq. non-linearities (order-preserving atomicMax).
__global__ void __launch_bounds__(256) reduce_slices_kernel(const float *__restrict__ partial,
                                                            int n_splits, size_t cells,
                                                            float inv_scale,
                                                            float *__restrict__ heat,
                                                            unsigned *__restrict__ maxima)
{
    float mx[2] = {-INFINITY, -INFINITY};
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < 2 * cells;
         q += (size_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int sp = 0; sp < n_splits; ++sp) s += partial[(size_t)sp * 2 * cells + q];
        s *= inv_scale;
        heat[q] = s;
        int c = q < cells ? 0 : 1;
        mx[c] = fmaxf(mx[c], s);
    }
    for (int c = 0; c < 2; ++c) {
        float m = mx[c];
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0 && m > -INFINITY) atomicMax(&maxima[c], float_to_ordered(m));
    }
}

// P -> P_hat = (P / m)^2 (Eq. non-linearities), 0 where the class maximum m is
// not positive; the decode_mode toggles switch the division or the square off.
__global__ void nonlinear_kernel(float *__restrict__ heat, size_t cells,
                                 const unsigned *__restrict__ maxima, unsigned mode)
{
    const float m0 = ordered_to_float(maxima[0]), m1 = ordered_to_float(maxima[1]);
    const float i0 = m0 > 0.f ? 1.0f / m0 : 0.f, i1 = m1 > 0.f ? 1.0f / m1 : 0.f;
    const bool norm = !(mode & VSAOGM_MODE_NO_NORM), square = !(mode & VSAOGM_MODE_NO_SQUARE);
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < 2 * cells;
         q += (size_t)gridDim.x * blockDim.x) {
        float v = heat[q];
        if (norm) v *= q < cells ? i0 : i1;
        heat[q] = square ? v * v : v;
    }
}

// ---- batched forms (many maps per launch) ----
__global__ void __launch_bounds__(kNormThreads) norms_batch_kernel(const __grid_constant__ BatchNormTable tab)
{
    const int gs = blockIdx.x;
    int lo = 0, hi = tab.n_maps - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tab.m[mid].mem_begin <= gs) lo = mid; else hi = mid - 1;
    }
    const BatchNormMap &M = tab.m[lo];
    const int s = gs - M.mem_begin;
    const float t = norm2_row(M.omega + (size_t)s * M.D, M.D);
    if (threadIdx.x == 0) M.inv_norm[s] = t > 0.f ? rsqrtf(t) : 0.f;
}

__global__ void zero_maxima_batch_kernel(const __grid_constant__ BatchOutTable tab)
{
    const int i = threadIdx.x;
    if (i < tab.n_maps) {
        tab.m[i].maxima[0] = 0u;
        tab.m[i].maxima[1] = 0u;
    }
}

// blockIdx.y is the map: its slices summed in order, scaled, and the maxima.
// One block of kSumBlockOutputs outputs of one map per CTA (maps' blocks
// numbered one after the other, so large and small maps share the GPU evenly).
__global__ void __launch_bounds__(256) reduce_slices_batch_kernel(const __grid_constant__ BatchOutTable tab)
{
    const int qb = blockIdx.x;
    int lo = 0, hi = tab.n_maps - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tab.m[mid].sum_begin <= qb) lo = mid; else hi = mid - 1;
    }
    const BatchMapOut &M = tab.m[lo];
    const size_t cells = (size_t)M.W * M.H;
    const size_t q0 = (size_t)(qb - M.sum_begin) * kSumBlockOutputs;
    const size_t q1 = min(2 * cells, q0 + kSumBlockOutputs);
    float mx[2] = {-INFINITY, -INFINITY};
    for (size_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        float s = 0.f;
        for (int sp = 0; sp < M.splits; ++sp) s += M.partial[(size_t)sp * 2 * cells + q];
        s *= M.inv_scale;
        M.heat[q] = s;
        int c = q < cells ? 0 : 1;
        mx[c] = fmaxf(mx[c], s);
    }
    for (int c = 0; c < 2; ++c) {
        float m = mx[c];
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0 && m > -INFINITY) atomicMax(&M.maxima[c], float_to_ordered(m));
    }
}

__global__ void add_kernel(float2 *__restrict__ dst, const float2 *__restrict__ src, size_t n)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x) {
        float2 a = dst[q], b = src[q];
        dst[q] = make_float2(a.x + b.x, a.y + b.y);
    }
}

}  // namespace

int memory_norms(vsaogm_map *m, cudaStream_t st)
{
    StageScope sc(m, VSAOGM_STAGE_NORMS, st);
    norms_kernel<<<m->S, kNormThreads, 0, st>>>(m->omega, m->cfg.D, m->inv_norm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "decode: norms");
    sc.end(1);
    return VSAOGM_OK;
}

void region_blocks(const vsaogm_map *m, Region r, int bi, int bj, std::vector<DecodeBlock> &out)
{
    out.clear();
    const int tx = m->cfg.tiles_x, ty = m->cfg.tiles_y;
    for (int by = 0; by < ty; ++by) {
        const int y0 = std::max(r.y0, m->tile_first[1][by]), y1 = std::min(r.y1, m->tile_last[1][by]);
        if (y0 >= y1) continue;
        for (int bx = 0; bx < tx; ++bx) {
            const int x0 = std::max(r.x0, m->tile_first[0][bx]);
            const int x1 = std::min(r.x1, m->tile_last[0][bx]);
            if (x0 >= x1) continue;
            for (int j0 = y0; j0 < y1; j0 += bj)
                for (int i0 = x0; i0 < x1; i0 += bi)
                    out.push_back(DecodeBlock{by * tx + bx, i0, j0, std::min(i0 + bi, x1),
                                              std::min(j0 + bj, y1)});
        }
    }
}

int decode_region(vsaogm_map *m, Region r, float *heat, cudaStream_t st)
{
    int rc = memory_norms(m, st);
    if (rc) return rc;
    if (m->cfg.decode_prec != VSAOGM_DECODE_FP32) return decode_tensor_cores(m, r, heat, st);
    std::vector<DecodeBlock> blocks;
    region_blocks(m, r, kBI, kBJ, blocks);
    const int D = m->cfg.D, nb = (int)blocks.size();
    const size_t cells = (size_t)r.w() * r.h();
    // slices of the frequencies: about three resident CTAs per SM in total
    int splits = std::max(1, std::min((D + kKC - 1) / kKC, 3 * 152 / std::max(nb, 1)));
    const int kps = ((D + splits - 1) / splits + kKC - 1) / kKC * kKC;
    splits = (D + kps - 1) / kps;
    rc = ensure(m->ws.dec_partial, sizeof(float) * (size_t)splits * 2 * cells);
    if (rc) return rc;
    StageScope sc(m, VSAOGM_STAGE_DECODE, st);
    const OutGeom og{r.x0, r.y0, r.w(), r.h()};
    int launches = 0;
    for (int b0 = 0; b0 < nb; b0 += kMaxLaunchBlocks) {
        BlockBatch batch;
        batch.n = std::min(kMaxLaunchBlocks, nb - b0);
        for (int q = 0; q < batch.n; ++q) batch.b[q] = blocks[b0 + q];
        decode_fp32_kernel<<<dim3(batch.n, splits), 256, 0, st>>>(
            batch, m->omega, m->inv_norm, m->nu, D, og, m->col_off, m->row_off, kps,
            (float *)m->ws.dec_partial.ptr);
        ++launches;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "decode: fp32");
    if ((rc = sum_slices(m, (const float *)m->ws.dec_partial.ptr, splits, cells, 1.0f, heat, st)))
        return rc;
    sc.end(launches + 1);
    return VSAOGM_OK;
}

// Grows the decode scratch so that no map or window query allocates.  A query
// of a region with nb blocks uses at most (slots / nb) frequency slices, and the
// blocks cover the region, so slices x cells <= slots x block cells: 152 x 256 x 128
// for the tensor-core decode, 456 x 64^2 for the SIMT one; the tensor-core
// decode's minimum of ceil(D / kTcMaxKPerSplit) slices of the whole map (or
// one slice) bounds the rest.
int reserve_decode(vsaogm_map *m)
{
    const size_t cells = (size_t)m->cfg.grid_w * m->cfg.grid_h;
    const size_t tc_slices = (size_t)(m->cfg.D + kTcMaxKPerSplit - 1) / kTcMaxKPerSplit;
    size_t need = std::max<size_t>(
        {(size_t)152 * 256 * 128, (size_t)3 * 152 * kBI * kBJ, tc_slices * cells});
    return ensure(m->ws.dec_partial, sizeof(float) * 2 * need);
}

int sum_slices(vsaogm_map *m, const float *partial, int splits, size_t cells, float inv_scale,
               float *heat, cudaStream_t st)
{
    // ordered encoding 0 is below every float: the running maximum starts empty
    cudaError_t e = cudaMemsetAsync(m->maxima, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_error(e, "decode");
    int blocks = (int)std::min<size_t>((2 * cells + 255) / 256, 152 * 8);
    reduce_slices_kernel<<<blocks, 256, 0, st>>>(partial, splits, cells, inv_scale, heat,
                                                 m->maxima);
    e = cudaGetLastError();
    return e == cudaSuccess ? VSAOGM_OK : cuda_error(e, "decode: slice sum");
}

int apply_nonlinearity(vsaogm_map *m, float *heat, cudaStream_t st, size_t cells)
{
    StageScope sc(m, VSAOGM_STAGE_NONLINEAR, st);
    if (cells == 0) cells = (size_t)m->cfg.grid_w * m->cfg.grid_h;
    int blocks = (int)std::min<size_t>((2 * cells + 255) / 256, 152 * 16);
    nonlinear_kernel<<<blocks, 256, 0, st>>>(heat, cells, m->maxima, m->cfg.decode_mode);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "decode: non-linearity");
    sc.end(1);
    return VSAOGM_OK;
}

int launch_norms_batch(const BatchNormTable &tab, int total_memories, cudaStream_t st)
{
    norms_batch_kernel<<<total_memories, kNormThreads, 0, st>>>(tab);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VSAOGM_OK : cuda_error(e, "batch norms");
}

int launch_sums_batch(const BatchOutTable &tab, int total_blocks, cudaStream_t st)
{
    zero_maxima_batch_kernel<<<1, kMaxBatchMaps, 0, st>>>(tab);
    if (total_blocks > 0) reduce_slices_batch_kernel<<<total_blocks, 256, 0, st>>>(tab);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VSAOGM_OK : cuda_error(e, "batch slice sums");
}

int add_memories(float2 *dst, const float2 *src, int64_t count, cudaStream_t st)
{
    int blocks = (int)std::min<int64_t>((count + 255) / 256, 152 * 16);
    add_kernel<<<blocks, 256, 0, st>>>(dst, src, (size_t)count);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VSAOGM_OK : cuda_error(e, "fuse");
}

VSAOGM_CHECK_TU(decode)

}  // namespace vsaogm_impl
