// Decoding on the 5th-generation tensor cores (Eq. loc-query, split precision).
//
// For one block of up to 128 rows (y cells) x N columns (x cells) inside one
// tile, and a slice of the frequencies k, both class maps are the real GEMM
//   P_psi[m][n] = sum_k' Aop_psi[m][k'] * Bop[n][k'],
//   Aop_psi[m][2k] = Re U_psi(j_m, k),  Aop_psi[m][2k+1] = -Im U_psi(j_m, k),
//   Bop[n][2k]     = Re A(i_n, k),      Bop[n][2k+1]     =  Im A(i_n, k),
// with A(i, k) = exp(i 2 pi nu_x[k] dx_i) and U_psi = conj(w_hat_psi[k]) *
// exp(i 2 pi nu_y[k] dy_j): the sum over k' is Re sum_k U A, i.e. Eq. loc-query
// in its separable form.  Both operands are generated in shared memory (sin/cos
// after an exact phase reduction, then the complex product), never read from
// HBM, in the 128-byte-swizzled K-major layout the tensor cores read.
//
// Precision: each operand is split x = hi + lo in BF16 (or FP16, with U scaled
// by a power of two to stay clear of FP16 subnormals) and the product is
// hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory: about 16
// significant bits per product.
//
// Blocks: up to 128 columns inside one tile column by up to 128 rows that may
// cross tile rows (each row multiplies the memories of its own tile), so the
// 128-row MMA tile is filled even when tiles are short.
//
// Pipeline per CTA (512 threads, one CTA per SM): all threads generate stage s
// (32 frequencies) into one of two shared-memory buffers while the tensor
// cores run stage s - 1 from the other; the memories and frequencies of stage
// s + 1 are loaded into registers meanwhile.  One thread issues the 24 MMAs
// of a stage (2 classes x 3 products x 4 K-steps of 16) and commits them to
// the buffer's mbarrier.  The 128-byte swizzle puts 4-byte element kk of row
// m at byte m * 128 + ((kk / 4) xor (m mod 8)) * 16 + (kk mod 4) * 4.  The epilogue reads the two 128 x N FP32 accumulators
// from tensor memory and writes per-slice partial maps; a second kernel sums
// the slices in a fixed order and folds the per-class maxima (Eq.
// non-linearities needs the map maximum).  Every wait is bounded: on time-out
// the CTA records VSAOGM_E_TIMEOUT, drains its MMAs, frees its tensor memory
// and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "internal.cuh"
#include "sm100.cuh"

namespace vsaogm_impl {
namespace {

using namespace sm100;

constexpr int kM = 128;            // rows per block (MMA M)
constexpr int kKS = 32;            // frequencies per stage (64 k' = 128 bytes per row)
constexpr int kRowBytes = 128;
constexpr int kProducers = 512;    // 16 warps generate the operands ...
constexpr int kWarps = kProducers / 32;
constexpr int kThreads = kProducers + 32;  // ... and one more issues the MMAs
constexpr int kQ = kM / kWarps;    // rows (and columns) per thread
constexpr int kATile = kM * kRowBytes;          // one A operand tile (16 KB)
constexpr int kAStage = 4 * kATile;             // 2 classes x hi/lo (64 KB)
constexpr int kWBytes = kMaxBlockTiles * 2 * kKS * 8;  // staged memories (8 KB)
constexpr int kWPerThread = (kMaxBlockTiles * 2 * kKS + kProducers - 1) / kProducers;
constexpr int kTmemCols = 256;                  // class psi accumulates at column 128 psi
constexpr uint64_t kWaitNs = 2000000000ull;     // 2 s: far above any legitimate wait

// Bytes of one pipeline stage for MMA width N: A (both classes, hi and lo),
// B (hi and lo) and the staged memories.
__host__ __device__ constexpr int stage_size(int N) { return kAStage + 2 * N * kRowBytes + kWBytes; }
constexpr size_t kSmemMax = 1024 + 2 * (size_t)stage_size(kM);

__device__ __forceinline__ float2 phasor(float nu, float d)
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

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <bool BF16>
__device__ __forceinline__ void split2(float x, float y, uint32_t &hi, uint32_t &lo)
{
    if (BF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
        const uint32_t hb = *reinterpret_cast<uint32_t *>(&h);
        // bf16 -> f32 is a shift of the bit pattern; both residuals in one packed sub
        const f32x2 hf = pack2(__uint_as_float(hb << 16), __uint_as_float(hb & 0xffff0000u));
        const float2 d = unpack2(sub2(pack2(x, y), hf));
        __nv_bfloat162 l = __floats2bfloat162_rn(d.x, d.y);
        hi = hb;
        lo = *reinterpret_cast<uint32_t *>(&l);
    } else {
        __half2 h = __floats2half2_rn(x, y);
        float2 hf = __half22float2(h);
        __half2 l = __floats2half2_rn(x - hf.x, y - hf.y);
        hi = *reinterpret_cast<uint32_t *>(&h);
        lo = *reinterpret_cast<uint32_t *>(&l);
    }
}

// One (block of cells, frequency slice) item, executed by the whole CTA:
// kProducers threads (16 warps) generate the operands, one more warp issues
// the MMAs.  The block's columns lie in tile column b.tile; its rows may cross
// tile rows (at most kMaxBlockTiles of them), each row using the memories of
// its own tile: row j of the A operand is U_psi of tile (row_tile[j], b.tile).
//
// Hand-offs: producers arrive on full_bar[buf] (one arrival per warp, after
// each thread's proxy fence) when stage s is in buffer buf = s & 1; the MMA
// warp waits on it, issues the stage's 24 MMAs and commits them to
// empty_bar[buf], which producers wait on before refilling buf at stage s + 2.
// Producers also meet at named barrier 1 once per stage, because each stage's
// memories are staged by all of them for all of them.  Every wait is bounded;
// after a time-out the CTA stops waiting, records VSAOGM_E_TIMEOUT, drains
// and frees its tensor memory.
template <bool BF16>
__device__ __forceinline__ void decode_tc_body(
    const DecodeBlock b, const int split, const float2 *__restrict__ omega,
    const float *__restrict__ inv_norm, const float *__restrict__ nu, int D, int tiles_x,
    const int *__restrict__ row_tile, OutGeom og, const float *__restrict__ col_off,
    const float *__restrict__ row_off, float res, int k_per_split, int N, float u_scale,
    float *__restrict__ partial, int *__restrict__ status)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[2], empty_bar[2], done_bar;
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;
    volatile int *abort_v = &abort_s;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int stage_bytes = stage_size(N);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int k_begin = split * k_per_split;
    const int k_end = min(D, k_begin + k_per_split);
    const int n_stages = (k_end - k_begin + kKS - 1) / kKS;
    const int ni = b.i1 - b.i0, nj = b.j1 - b.j0;
    const int by0 = row_tile[b.j0];
    const int nt = row_tile[b.j1 - 1] - by0 + 1;  // tile rows of the block
    if (nt < 1 || nt > kMaxBlockTiles || N > kM || N < 16 || (N & 15)) {
        // the host never builds such a block; refuse it rather than index past smem
        if (tid == 0) atomicExch(status, VSAOGM_E_INVAL);
        return;
    }

    if (warp == 0) {
        tmem_alloc(&tmem_base_s, kTmemCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&full_bar[0], kWarps);
        mbar_init(&full_bar[1], kWarps);
        mbar_init(&empty_bar[0], 1);
        mbar_init(&empty_bar[1], 1);
        mbar_init(&done_bar, 1);
        mbar_fence_init();
        abort_s = 0;
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = tmem_base_s;

    if (warp == kWarps) {
        // ------------------------------------------------------ MMA warp
        const uint32_t idesc = idesc_f16(kM, N, BF16);
        for (int s = 0; s < n_stages; ++s) {
            const int buf = s & 1;
            if (!*abort_v && !mbar_wait(&full_bar[buf], (uint32_t)(s >> 1) & 1u, kWaitNs))
                atomicExch(&abort_s, 1);
            tc_fence_after_sync();
            if (lane == 0) {
                uint8_t *st = smem + (size_t)buf * stage_bytes;
                const uint32_t a0 = smem_addr(st), bhi = smem_addr(st + kAStage);
                const uint32_t blo = bhi + (uint32_t)(N * kRowBytes);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t off = kk * 32;  // 16 elements of 2 bytes
                    const uint64_t dbh = desc_k_sw128(bhi + off), dbl = desc_k_sw128(blo + off);
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const uint64_t dah = desc_k_sw128(a0 + (2 * c) * kATile + off);
                        const uint64_t dal = desc_k_sw128(a0 + (2 * c + 1) * kATile + off);
                        const uint32_t d = tmem + 128u * c;
                        mma_f16(d, dah, dbh, idesc, (s > 0 || kk > 0) ? 1u : 0u);
                        mma_f16(d, dah, dbl, idesc, 1u);
                        mma_f16(d, dal, dbh, idesc, 1u);
                    }
                }
                mma_commit(&empty_bar[buf]);
            }
            __syncwarp();
        }
        // one more commit arrives when every MMA issued above has finished
        if (lane == 0) mma_commit(&done_bar);
        __syncwarp();
    } else {
        // ------------------------------------------------------ producers
        // Fixed per-thread geometry: frequency kk = lane; rows / columns
        // warp + kWarps q, whose 128-byte swizzle phase (row & 7) is warp & 7.
        float dy[kQ], dx[kQ];
        int tl[kQ];  // tile row of each A row, relative to by0
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const int m = warp + kWarps * q;
            dy[q] = m < nj ? row_off[b.j0 + m] : 0.f;
            tl[q] = m < nj ? min(max(row_tile[b.j0 + m] - by0, 0), nt - 1) : 0;
            dx[q] = m < ni ? col_off[b.i0 + m] : 0.f;
        }
        const uint32_t soff = (uint32_t)(warp * kRowBytes +
                                         ((((lane >> 2) ^ (warp & 7)) << 4) | ((lane & 3) << 2)));
        // The memories of a stage's 32 frequencies for the block's tiles are
        // staged (scaled by 1 / norm) in the stage buffer's W area: entry
        // e = (tile row, class, kk), kWPerThread entries per thread.
        int w_mem[kWPerThread];
        float w_scale[kWPerThread];
#pragma unroll
        for (int r = 0; r < kWPerThread; ++r) {
            const int e = tid + kProducers * r;
            const bool ev = e < nt * 2 * kKS;
            const int mem = 2 * ((by0 + (e >> 6)) * tiles_x + b.tile) + ((e >> 5) & 1);
            w_mem[r] = ev ? mem : -1;
            w_scale[r] = ev ? inv_norm[mem] * u_scale : 0.f;
        }
        // prefetch registers: this thread's frequency and staged memory entries
        float pnx = 0.f, pny = 0.f;
        float2 pw[kWPerThread];
        auto prefetch = [&](int s) {
            const int k = k_begin + s * kKS + lane;
            pnx = k < k_end ? nu[k] : 0.f;
            pny = k < k_end ? nu[D + k] : 0.f;
#pragma unroll
            for (int r = 0; r < kWPerThread; ++r) {
                const int kk = k_begin + s * kKS + ((tid + kProducers * r) & 31);
                pw[r] = (w_mem[r] >= 0 && kk < k_end) ? omega[(size_t)w_mem[r] * D + kk]
                                                       : make_float2(0.f, 0.f);
            }
        };
        // the memories of stage s go to the W area of buffer s & 1 (no MMA reads it)
        auto stage_w = [&](int s) {
            float2 *sw = reinterpret_cast<float2 *>(smem + (size_t)(s & 1) * stage_bytes +
                                                    kAStage + 2 * N * kRowBytes);
#pragma unroll
            for (int r = 0; r < kWPerThread; ++r)
                if (w_mem[r] >= 0)
                    sw[tid + kProducers * r] =
                        make_float2(pw[r].x * w_scale[r], pw[r].y * w_scale[r]);
        };
        if (n_stages > 0) {
            prefetch(0);
            stage_w(0);
        }
        float nux = pnx, nuy = pny;
        named_bar_sync(1, kProducers);
        uint32_t phase_bits = 0u;  // bit b: parity to wait for on empty_bar[b]
        const float step_d = kWarps * res;  // offset between a thread's consecutive rows / columns

        for (int s = 0; s < n_stages; ++s) {
            const int buf = s & 1;
            if (s >= 2) {
                if (!*abort_v && !mbar_wait(&empty_bar[buf], (phase_bits >> buf) & 1u, kWaitNs))
                    atomicExch(&abort_s, 1);
                phase_bits ^= 1u << buf;
            }
            uint8_t *st = smem + (size_t)buf * stage_bytes;
            uint8_t *bh = st + kAStage, *bl = bh + N * kRowBytes;
            const float2 *sw = reinterpret_cast<const float2 *>(bl + N * kRowBytes);
            const bool kv = k_begin + s * kKS + lane < k_end;
            if (s + 1 < n_stages) prefetch(s + 1);  // in flight while this stage is generated
            // B operand: x phasors of the N columns.  Column warp + 16 (q + 1)
            // is 16 cells right of column warp + 16 q in the same tile, so its
            // phasor is the previous one times exp(i 2 pi nu_x 16 res).
            {
                const float2 rot = phasor(nux, step_d);
                float2 a = phasor(nux, dx[0]);
#pragma unroll
                for (int q = 0; q < kQ; ++q) {
                    const int n = warp + kWarps * q;
                    if (n >= N) break;
                    if (q > 0) a = cmul(a, rot);
                    const float2 v = (kv && n < ni) ? a : make_float2(0.f, 0.f);
                    uint32_t hi, lo;
                    split2<BF16>(v.x, v.y, hi, lo);
                    *reinterpret_cast<uint32_t *>(bh + q * kWarps * kRowBytes + soff) = hi;
                    *reinterpret_cast<uint32_t *>(bl + q * kWarps * kRowBytes + soff) = lo;
                }
            }
            // A operands: U_psi = conj(w_hat_psi) * y phasor, stored as
            // (Re, -Im).  Rows step by 16 cells too, except where a row enters
            // the next tile (warp-uniform): there the phasor and the memories
            // are reloaded.
            {
                const float2 rot = phasor(nuy, step_d);
                float2 e = phasor(nuy, dy[0]);
                float2 w0 = sw[(2 * tl[0]) * kKS + lane], w1 = sw[(2 * tl[0] + 1) * kKS + lane];
#pragma unroll
                for (int q = 0; q < kQ; ++q) {
                    const int m = warp + kWarps * q;
                    if (q > 0) {
                        if (tl[q] != tl[q - 1]) {
                            e = phasor(nuy, dy[q]);
                            w0 = sw[(2 * tl[q]) * kKS + lane];
                            w1 = sw[(2 * tl[q] + 1) * kKS + lane];
                        } else {
                            e = cmul(e, rot);
                        }
                    }
                    const float2 v = (kv && m < nj) ? e : make_float2(0.f, 0.f);
                    float u0r = w0.x * v.x + w0.y * v.y, u0i = w0.x * v.y - w0.y * v.x;
                    float u1r = w1.x * v.x + w1.y * v.y, u1i = w1.x * v.y - w1.y * v.x;
                    const uint32_t o = q * kWarps * kRowBytes + soff;
                    uint32_t hi, lo;
                    split2<BF16>(u0r, -u0i, hi, lo);
                    *reinterpret_cast<uint32_t *>(st + 0 * kATile + o) = hi;
                    *reinterpret_cast<uint32_t *>(st + 1 * kATile + o) = lo;
                    split2<BF16>(u1r, -u1i, hi, lo);
                    *reinterpret_cast<uint32_t *>(st + 2 * kATile + o) = hi;
                    *reinterpret_cast<uint32_t *>(st + 3 * kATile + o) = lo;
                }
            }
            // hand the stage to the MMA warp
            fence_async_shared();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full_bar[buf]);
            // the next stage's memories into the other buffer's W area (its
            // readers finished before the previous producer barrier)
            if (s + 1 < n_stages) {
                stage_w(s + 1);
                nux = pnx;
                nuy = pny;
            }
            named_bar_sync(1, kProducers);
        }
    }
    // epilogue (producers): warp w reads TMEM lanes 32 (w & 3) .. + 31 (its lane
    // quarter), class (w >> 2) & 1, and one half of the 16-column chunks (w >> 3)
    // always drain (bounded), even after a time-out: tensor memory is freed below
    if (!mbar_wait(&done_bar, 0u, kWaitNs)) atomicExch(&abort_s, 1);
    tc_fence_after_sync();
    __syncthreads();
    if (warp < kWarps) {
        const int c = (warp >> 2) & 1, lane_base = 32 * (warp & 3), half = warp >> 3;
        const int m = lane_base + lane;
        const int nch = N / 16, ch0 = half ? (nch + 1) / 2 : 0, ch1 = half ? nch : (nch + 1) / 2;
        float *out = partial + (((size_t)split * 2 + c) * og.OH) * og.OW;
        if (!abort_s && n_stages > 0) {
            for (int cc = ch0; cc < ch1; ++cc) {
                float v[16];
                tmem_ld_32x32b_x16(tmem + ((uint32_t)lane_base << 16) + 128u * c + cc * 16, v);
                if (m < nj) {
                    float *row = out + (size_t)(b.j0 + m - og.oy) * og.OW + (b.i0 - og.ox);
#pragma unroll
                    for (int x = 0; x < 16; ++x)
                        if (cc * 16 + x < ni) row[cc * 16 + x] = v[x];
                }
            }
        } else if (!abort_s && n_stages == 0) {
            // no frequencies in this slice: its contribution is zero
            if (m < nj)
                for (int x = ch0 * 16; x < min(ni, ch1 * 16); ++x)
                    out[(size_t)(b.j0 + m - og.oy) * og.OW + (b.i0 - og.ox) + x] = 0.f;
        }
    }
    if (abort_s && tid == 0) atomicExch(status, VSAOGM_E_TIMEOUT);
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

template <bool BF16>
__global__ void __launch_bounds__(kThreads, 1) decode_tc_kernel(
    const BlockBatch blocks, const float2 *__restrict__ omega, const float *__restrict__ inv_norm,
    const float *__restrict__ nu, int D, int tiles_x, const int *__restrict__ row_tile, OutGeom og,
    const float *__restrict__ col_off, const float *__restrict__ row_off, float res,
    int k_per_split, int N, float u_scale, float *__restrict__ partial, int *__restrict__ status)
{
    decode_tc_body<BF16>(blocks.b[blockIdx.x], blockIdx.y, omega, inv_norm, nu, D, tiles_x,
                         row_tile, og, col_off, row_off, res, k_per_split, N, u_scale, partial,
                         status);
}

// Many maps in one launch: CTA q decodes item q of a device list of
// (map, block, slice); each map's pointers come from the table.
template <bool BF16>
__global__ void __launch_bounds__(kThreads, 1) decode_tc_batch_kernel(
    const __grid_constant__ BatchDecodeTable tab, const BatchDecodeItem *__restrict__ items)
{
    const BatchDecodeItem it = items[blockIdx.x];
    const BatchDecodeMap &M = tab.m[it.map];
    const int N = ((it.b.i1 - it.b.i0) + 15) / 16 * 16;
    decode_tc_body<BF16>(it.b, it.split, M.omega, M.inv_norm, M.nu, M.D, M.tiles_x, M.row_tile,
                         OutGeom{0, 0, M.W, M.H}, M.col_off, M.row_off, M.res,
                         M.k_per_split, N, M.u_scale, M.partial, M.status);
}

}  // namespace

// Blocks of at most 128 x 128 cells covering region r for the tensor-core
// decode: columns inside one tile column, rows across at most kMaxBlockTiles
// tile rows.
void tc_blocks(const vsaogm_map *m, Region r, std::vector<DecodeBlock> &out)
{
    out.clear();
    const std::vector<int> &yl = m->tile_last[1];  // tiles are monotonic in the row index
    const int ty = m->cfg.tiles_y;
    for (int bx = 0; bx < m->cfg.tiles_x; ++bx) {
        const int x0 = std::max(r.x0, m->tile_first[0][bx]);
        const int x1 = std::min(r.x1, m->tile_last[0][bx]);
        if (x0 >= x1) continue;
        for (int i0 = x0; i0 < x1; i0 += kM) {
            const int i1 = std::min(i0 + kM, x1);
            int by = 0;
            for (int j0 = r.y0; j0 < r.y1;) {
                while (by < ty - 1 && yl[by] <= j0) ++by;  // tile row of row j0
                // rows up to the end of the kMaxBlockTiles-th tile row from by
                int cap = j0 + 1;
                for (int t = by; t < std::min(by + kMaxBlockTiles, ty); ++t) cap = std::max(cap, yl[t]);
                const int j1 = std::min({j0 + kM, r.y1, cap});
                out.push_back(DecodeBlock{bx, i0, j0, i1, j1});
                j0 = j1;
            }
        }
    }
}

int launch_decode_tc_batch(const BatchDecodeTable &tab, const BatchDecodeItem *items,
                           int n_items, bool bf16, cudaStream_t st)
{
    cudaError_t e;
    if (bf16) {
        e = cudaFuncSetAttribute(decode_tc_batch_kernel<true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
        if (e == cudaSuccess)
            decode_tc_batch_kernel<true><<<n_items, kThreads, kSmemMax, st>>>(tab, items);
    } else {
        e = cudaFuncSetAttribute(decode_tc_batch_kernel<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
        if (e == cudaSuccess)
            decode_tc_batch_kernel<false><<<n_items, kThreads, kSmemMax, st>>>(tab, items);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? VSAOGM_OK : cuda_error(e, "batch decode");
}

float tc_u_scale(const vsaogm_map *m)
{
    float u = 1.f;
    if (m->cfg.decode_prec == VSAOGM_DECODE_FP16X3)
        while (u * u * 4.f <= (float)m->cfg.D) u *= 2.f;
    return u;
}

int decode_tensor_cores(vsaogm_map *m, Region r, float *heat, cudaStream_t st)
{
    const int D = m->cfg.D;
    const bool bf16 = m->cfg.decode_prec == VSAOGM_DECODE_BF16X3;
    std::vector<DecodeBlock> blocks;
    tc_blocks(m, r, blocks);
    const int nb = (int)blocks.size();
    // slices of the frequencies so that blocks x slices fills the 152 SMs once,
    // and no slice longer than kTcMaxKPerSplit
    int splits = std::max((D + kTcMaxKPerSplit - 1) / kTcMaxKPerSplit,
                          std::min((D + kKS - 1) / kKS, 152 / std::max(nb, 1)));
    int kps = ((D + splits - 1) / splits + kKS - 1) / kKS * kKS;
    splits = (D + kps - 1) / kps;
    const size_t cells = (size_t)r.w() * r.h();
    int rc = ensure(m->ws.dec_partial, sizeof(float) * (size_t)splits * 2 * cells);
    if (rc) return rc;
    const float u_scale = tc_u_scale(m);
    cudaError_t e = bf16 ? cudaFuncSetAttribute(decode_tc_kernel<true>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)kSmemMax)
                         : cudaFuncSetAttribute(decode_tc_kernel<false>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)kSmemMax);
    if (e != cudaSuccess) return cuda_error(e, "decode: tensor cores");
    StageScope sc(m, VSAOGM_STAGE_DECODE, st);
    float *part = (float *)m->ws.dec_partial.ptr;
    const OutGeom og{r.x0, r.y0, r.w(), r.h()};
    int launches = 0;
    for (int b0 = 0; b0 < nb; b0 += kMaxLaunchBlocks) {
        BlockBatch batch;
        batch.n = std::min(kMaxLaunchBlocks, nb - b0);
        int widest = 16;
        for (int q = 0; q < batch.n; ++q) {
            batch.b[q] = blocks[b0 + q];
            widest = std::max(widest, batch.b[q].i1 - batch.b[q].i0);
        }
        const int N = (widest + 15) / 16 * 16;  // MMA N: the widest block, multiple of 16
        const size_t smem = 1024 + 2 * (size_t)stage_size(N);
        dim3 grid(batch.n, splits);
        if (bf16)
            decode_tc_kernel<true><<<grid, kThreads, smem, st>>>(
                batch, m->omega, m->inv_norm, m->nu, D, m->cfg.tiles_x, m->row_tile, og,
                m->col_off, m->row_off, m->cfg.resolution, kps, N, u_scale, part, m->status);
        else
            decode_tc_kernel<false><<<grid, kThreads, smem, st>>>(
                batch, m->omega, m->inv_norm, m->nu, D, m->cfg.tiles_x, m->row_tile, og,
                m->col_off, m->row_off, m->cfg.resolution, kps, N, u_scale, part, m->status);
        ++launches;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "decode: tensor cores");
    if ((rc = sum_slices(m, part, splits, cells, 1.0f / u_scale, heat, st))) return rc;
    sc.end(launches + 1);
    return VSAOGM_OK;
}

}  // namespace vsaogm_impl
