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
// Pipeline per CTA (256 threads, one CTA per SM): all threads generate stage s
// (32 frequencies) into one of two shared-memory buffers while the tensor
// cores run stage s - 1 from the other; one thread issues the 24 MMAs of a
// stage (2 classes x 3 products x 4 K-steps of 16) and commits them to the
// buffer's mbarrier.  The epilogue reads the two 128 x N FP32 accumulators
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
constexpr int kATile = kM * kRowBytes;          // one A operand tile (16 KB)
constexpr int kAStage = 4 * kATile;             // 2 classes x hi/lo (64 KB)
constexpr int kTmemCols = 256;                  // class psi accumulates at column 128 psi
constexpr uint64_t kWaitNs = 2000000000ull;     // 2 s: far above any legitimate wait

__device__ __forceinline__ uint32_t swz(int row, int kk)
{
    // byte offset of the 4-byte element kk (0..31) of a 128-byte row, 128B swizzle
    return (uint32_t)(row * kRowBytes + ((((kk >> 2) ^ (row & 7)) << 4) | ((kk & 3) << 2)));
}

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

template <bool BF16>
__device__ __forceinline__ void split2(float x, float y, uint32_t &hi, uint32_t &lo)
{
    if (BF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
        float2 hf = __bfloat1622float2(h);
        __nv_bfloat162 l = __floats2bfloat162_rn(x - hf.x, y - hf.y);
        hi = *reinterpret_cast<uint32_t *>(&h);
        lo = *reinterpret_cast<uint32_t *>(&l);
    } else {
        __half2 h = __floats2half2_rn(x, y);
        float2 hf = __half22float2(h);
        __half2 l = __floats2half2_rn(x - hf.x, y - hf.y);
        hi = *reinterpret_cast<uint32_t *>(&h);
        lo = *reinterpret_cast<uint32_t *>(&l);
    }
}

// One (block of cells, frequency slice) item, executed by the whole CTA.
template <bool BF16>
__device__ __forceinline__ void decode_tc_body(
    const DecodeBlock b, const int split, const float2 *__restrict__ omega,
    const float *__restrict__ inv_norm, const float *__restrict__ nu, int D, OutGeom og,
    const float *__restrict__ col_off, const float *__restrict__ row_off, int k_per_split, int N,
    float u_scale, float *__restrict__ partial, int *__restrict__ status)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t empty_bar[2], done_bar;
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int stage_bytes = kAStage + 2 * N * kRowBytes;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int k_begin = split * k_per_split;
    const int k_end = min(D, k_begin + k_per_split);
    const int n_stages = (k_end - k_begin + kKS - 1) / kKS;
    const int ni = b.i1 - b.i0, nj = b.j1 - b.j0;

    if (warp == 0) {
        tmem_alloc(&tmem_base_s, kTmemCols);
        tmem_relinquish();
    }
    if (tid == 0) {
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

    // Fixed per-thread geometry: frequency kk = lane, rows / columns warp + 8q.
    float dy[kM / 8], dx[kM / 8];
#pragma unroll
    for (int q = 0; q < kM / 8; ++q) {
        int m = warp + 8 * q;
        dy[q] = m < nj ? row_off[b.j0 + m] : 0.f;
        dx[q] = m < ni ? col_off[b.i0 + m] : 0.f;
    }
    const float w0s = inv_norm[2 * b.tile] * u_scale, w1s = inv_norm[2 * b.tile + 1] * u_scale;
    const float2 *om0 = omega + (size_t)(2 * b.tile) * D;
    const float2 *om1 = om0 + D;
    const uint32_t idesc = idesc_f16(kM, N, BF16);
    uint32_t phase_bits = 0u;  // bit b: parity to wait for on buffer b

    for (int s = 0; s < n_stages; ++s) {
        const int buf = s & 1;
        if (s >= 2) {
            if (!mbar_wait(&empty_bar[buf], (phase_bits >> buf) & 1u, kWaitNs))
                atomicExch(&abort_s, 1);
            phase_bits ^= 1u << buf;
        }
        __syncthreads();
        if (abort_s) break;
        uint8_t *st = smem + (size_t)buf * stage_bytes;
        const int k = k_begin + s * kKS + lane;
        const bool kv = k < k_end;
        const float nux = kv ? nu[k] : 0.f, nuy = kv ? nu[D + k] : 0.f;
        float2 w0 = kv ? om0[k] : make_float2(0.f, 0.f);
        float2 w1 = kv ? om1[k] : make_float2(0.f, 0.f);
        w0.x *= w0s; w0.y *= w0s;
        w1.x *= w1s; w1.y *= w1s;
        // B operand: x phasors of the N columns
        uint8_t *bh = st + kAStage, *bl = bh + N * kRowBytes;
#pragma unroll
        for (int q = 0; q < kM / 8; ++q) {
            int n = warp + 8 * q;
            if (n >= N) continue;
            float2 a = (kv && n < ni) ? phasor(nux, dx[q]) : make_float2(0.f, 0.f);
            uint32_t hi, lo;
            split2<BF16>(a.x, a.y, hi, lo);
            *reinterpret_cast<uint32_t *>(bh + swz(n, lane)) = hi;
            *reinterpret_cast<uint32_t *>(bl + swz(n, lane)) = lo;
        }
        // A operands: U_psi = conj(w_hat_psi) * y phasor, stored as (Re, -Im)
#pragma unroll
        for (int q = 0; q < kM / 8; ++q) {
            int m = warp + 8 * q;
            float2 e = (kv && m < nj) ? phasor(nuy, dy[q]) : make_float2(0.f, 0.f);
            float u0r = w0.x * e.x + w0.y * e.y, u0i = w0.x * e.y - w0.y * e.x;
            float u1r = w1.x * e.x + w1.y * e.y, u1i = w1.x * e.y - w1.y * e.x;
            uint32_t hi, lo;
            split2<BF16>(u0r, -u0i, hi, lo);
            *reinterpret_cast<uint32_t *>(st + 0 * kATile + swz(m, lane)) = hi;
            *reinterpret_cast<uint32_t *>(st + 1 * kATile + swz(m, lane)) = lo;
            split2<BF16>(u1r, -u1i, hi, lo);
            *reinterpret_cast<uint32_t *>(st + 2 * kATile + swz(m, lane)) = hi;
            *reinterpret_cast<uint32_t *>(st + 3 * kATile + swz(m, lane)) = lo;
        }
        fence_async_shared();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after_sync();
            const uint32_t a0 = smem_addr(st), bhi = smem_addr(bh), blo = smem_addr(bl);
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
    }
    // drain: one more commit arrives when every MMA issued above has finished
    if (tid == 0) mma_commit(&done_bar);
    bool ok = mbar_wait(&done_bar, 0u, kWaitNs);
    if (!ok) atomicExch(&abort_s, 1);
    tc_fence_after_sync();
    __syncthreads();
    if (!abort_s && n_stages > 0) {
        const int c = warp >> 2, lane_base = 32 * (warp & 3);
        const int m = lane_base + lane;
        float *out = partial + (((size_t)split * 2 + c) * og.OH) * og.OW;
        for (int cc = 0; cc < N / 16; ++cc) {
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
        const int c = warp >> 2, m = 32 * (warp & 3) + lane;
        float *out = partial + (((size_t)split * 2 + c) * og.OH) * og.OW;
        if (m < nj)
            for (int x = 0; x < ni; ++x)
                out[(size_t)(b.j0 + m - og.oy) * og.OW + (b.i0 - og.ox) + x] = 0.f;
    }
    if (abort_s && tid == 0) atomicExch(status, VSAOGM_E_TIMEOUT);
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

template <bool BF16>
__global__ void __launch_bounds__(256, 1) decode_tc_kernel(
    const BlockBatch blocks, const float2 *__restrict__ omega, const float *__restrict__ inv_norm,
    const float *__restrict__ nu, int D, OutGeom og, const float *__restrict__ col_off,
    const float *__restrict__ row_off, int k_per_split, int N, float u_scale,
    float *__restrict__ partial, int *__restrict__ status)
{
    decode_tc_body<BF16>(blocks.b[blockIdx.x], blockIdx.y, omega, inv_norm, nu, D, og, col_off,
                         row_off, k_per_split, N, u_scale, partial, status);
}

// Many maps in one launch: CTA q decodes item q of a device list of
// (map, block, slice); each map's pointers come from the table.
template <bool BF16>
__global__ void __launch_bounds__(256, 1) decode_tc_batch_kernel(
    const __grid_constant__ BatchDecodeTable tab, const BatchDecodeItem *__restrict__ items)
{
    const BatchDecodeItem it = items[blockIdx.x];
    const BatchDecodeMap &M = tab.m[it.map];
    const int N = ((it.b.i1 - it.b.i0) + 15) / 16 * 16;
    decode_tc_body<BF16>(it.b, it.split, M.omega, M.inv_norm, M.nu, M.D,
                         OutGeom{0, 0, M.W, M.H}, M.col_off, M.row_off, M.k_per_split, N,
                         M.u_scale, M.partial, M.status);
}

}  // namespace

int launch_decode_tc_batch(const BatchDecodeTable &tab, const BatchDecodeItem *items,
                           int n_items, bool bf16, cudaStream_t st)
{
    const size_t smem = 1024 + 2 * (size_t)(kAStage + 2 * 128 * kRowBytes);
    cudaError_t e;
    if (bf16) {
        e = cudaFuncSetAttribute(decode_tc_batch_kernel<true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) decode_tc_batch_kernel<true><<<n_items, 256, smem, st>>>(tab, items);
    } else {
        e = cudaFuncSetAttribute(decode_tc_batch_kernel<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) decode_tc_batch_kernel<false><<<n_items, 256, smem, st>>>(tab, items);
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
    region_blocks(m, r, 128, kM, blocks);
    const int nb = (int)blocks.size();
    // slices of the frequencies so that blocks x slices fills the 152 SMs once
    int splits = std::max(1, std::min((D + kKS - 1) / kKS, 152 / std::max(nb, 1)));
    int kps = ((D + splits - 1) / splits + kKS - 1) / kKS * kKS;
    splits = (D + kps - 1) / kps;
    const size_t cells = (size_t)r.w() * r.h();
    int rc = ensure(m->ws.dec_partial, sizeof(float) * (size_t)splits * 2 * cells);
    if (rc) return rc;
    float u_scale = 1.f;
    if (!bf16) {
        while (u_scale * u_scale * 4.f <= (float)D) u_scale *= 2.f;
    }
    const size_t smem_max = 1024 + 2 * (size_t)(kAStage + 2 * 128 * kRowBytes);
    cudaError_t e = bf16 ? cudaFuncSetAttribute(decode_tc_kernel<true>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem_max)
                         : cudaFuncSetAttribute(decode_tc_kernel<false>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem_max);
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
        const size_t smem = 1024 + 2 * (size_t)(kAStage + 2 * N * kRowBytes);
        dim3 grid(batch.n, splits);
        if (bf16)
            decode_tc_kernel<true><<<grid, 256, smem, st>>>(batch, m->omega, m->inv_norm, m->nu, D,
                                                            og, m->col_off, m->row_off, kps, N,
                                                            u_scale, part, m->status);
        else
            decode_tc_kernel<false><<<grid, 256, smem, st>>>(batch, m->omega, m->inv_norm, m->nu,
                                                             D, og, m->col_off, m->row_off, kps, N,
                                                             u_scale, part, m->status);
        ++launches;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "decode: tensor cores");
    if ((rc = sum_slices(m, part, splits, cells, 1.0f / u_scale, heat, st))) return rc;
    sc.end(launches + 1);
    return VSAOGM_OK;
}

}  // namespace vsaogm_impl
