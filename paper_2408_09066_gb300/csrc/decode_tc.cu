// Decoding on the 5th-generation tensor cores (Eq. loc-query, split precision).
//
// For one block of rows (y cells) x N columns (x cells) and a slice of the
// frequencies k, both class maps are the real GEMM
//   P_psi[m][n] = sum_k' Aop_psi[m][k'] * Bop[n][k'],
//   Aop_psi[m][2k] = Re U_psi(j_m, k),  Aop_psi[m][2k+1] = -Im U_psi(j_m, k),
//   Bop[n][2k]     = Re A(i_n, k),      Bop[n][2k+1]     =  Im A(i_n, k),
// with A(i, k) = exp(i 2 pi nu_x[k] dx_i) and U_psi = conj(w_hat_psi[k]) *
// exp(i 2 pi nu_y[k] dy_j): the sum over k' is Re sum_k U A, i.e. Eq. loc-query
// in its separable form.  The A operands depend on the memories and are
// generated in shared memory every call (sin/cos after an exact phase
// reduction for a thread's first row, a complex multiply by the map's 2-cell
// step phasor for the next ones, the product with the memories); the B operand
// depends only on the frequencies and the geometry, so it is computed once per
// map into an x-phasor table in HBM (already split, in the operand layout) and
// copied by TMA.  Both are read by the tensor cores in the 64-byte-swizzled
// K-major layout: word kk of row m at byte m * 64 + ((kk / 4) xor ((m / 2) mod
// 4)) * 16 + (kk mod 4) * 4.
//
// Precision: each operand is split x = hi + lo in BF16, FP16 or FP8 (e4m3) and
// the product is hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory:
// about 16 significant bits per product with BF16 or FP16, about 7 with FP8.
// U is scaled by a power of two for FP16 and FP8 to stay clear of their
// subnormals.  A 64-byte operand row (one pipeline stage) holds 16 complex
// frequencies in the 16-bit formats (kind::f16 MMAs) and 32 in FP8
// (kind::f8f6f4 MMAs).
//
// Blocks: in a tile column wider than 128 cells, one row block of up to 128
// rows by up to 256 columns (MMA N = 256); in a narrower one, two row blocks
// (up to 256 rows) by the tile column's width, sharing B.  Rows may cross tile
// rows (each row multiplies the memories of its own tile), so the 128-row MMA
// tiles are filled even when tiles are short.
//
// Pipeline per CTA (one CTA per SM): 16 producer warps generate the A operands
// of stage s into one of two buffers while the tensor cores run stage s - 1
// from the other; a loader warp stages the memories, frequencies and step
// phasors of each stage ahead of the producers; a TMA warp copies the B
// operand of each stage into a ring of four slots; an MMA warp issues the
// stage's MMAs (2 K-steps x row blocks x 2 classes x 3 products) and commits
// them to the buffers' mbarriers.  The warps hand stages over through
// mbarriers only.  The epilogue reads the FP32 accumulators from tensor memory
// in 16-column chunks, stages them in shared memory and writes per-slice
// partial maps in whole row segments; a second kernel sums the slices in a
// fixed order and folds the per-class maxima (Eq. non-linearities needs the
// map maximum).  Every wait is bounded: on time-out the CTA records
// VSAOGM_E_TIMEOUT, drains its MMAs and copies, frees its tensor memory and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "internal.cuh"
#include "sm100.cuh"

namespace vsaogm_impl {
namespace {

using namespace sm100;

enum TcPrec { kPrecBF16 = 0, kPrecFP16 = 1, kPrecFP8 = 2 };

constexpr int kM = 128;            // rows per row block (MMA M)
constexpr int kRowBytes = 64;      // bytes per operand row and stage (64-byte swizzle)
constexpr int kWords = kRowBytes / 4;  // 4-byte words per operand row
constexpr int kProducers = 512;    // 16 warps generate the A operands ...
constexpr int kWarps = kProducers / 32;
constexpr int kMmaWarp = kWarps;       // ... one issues the MMAs ...
constexpr int kLoadWarp = kWarps + 1;  // ... one stages each stage's inputs ...
constexpr int kBLoadWarp = kWarps + 2; // ... and one copies the B operand by TMA
constexpr int kThreads = kProducers + 96;
constexpr int kStep = 2;           // cells between a thread's consecutive rows
constexpr int kMaxRowBlocks = 2;   // 128-row blocks per CTA
constexpr int kMaxN = 256;         // MMA N of a one-row-block CTA (128 with two)
constexpr int kATile = kM * kRowBytes;           // one A operand tile (8 KB)
constexpr int kBoxRows = 64;       // rows of one TMA box of the x-phasor table
constexpr int kBRing = 4;          // B operand slots (TMA runs this many stages ahead)
constexpr int kTmemCols = 512;                   // accumulators: row blocks x classes x N
constexpr uint64_t kWaitNs = 2000000000ull;     // 2 s: far above any legitimate wait

// Frequencies per stage (one 64-byte operand row): 16 in the 16-bit formats
// (one complex value per word), 32 in FP8 (two per word).
__host__ __device__ constexpr int stage_freqs(int prec) { return prec == kPrecFP8 ? 32 : 16; }
__host__ __device__ constexpr int max_block_tiles(int) { return kMaxBlockTiles; }
// Bytes of the aux area of one stage: the staged memories (tile row, class,
// frequency) float2, then per frequency (nu_x, nu_y) and the x and y step
// phasors, float2 each; rounded up to 1024 bytes.
__host__ __device__ constexpr int aux_bytes(int prec)
{
    return ((max_block_tiles(prec) * 2 + 3) * stage_freqs(prec) * 8 + 1023) / 1024 * 1024;
}
// Shared memory of a CTA with rb row blocks and MMA width N: two A buffers
// (row blocks x classes x hi/lo tiles), two aux areas, then kBRing B slots of
// a hi and a lo tile of N rows rounded up to whole TMA boxes.  Every offset
// is a multiple of 1024 bytes.
__host__ __device__ constexpr int a_buffer_bytes(int rb) { return rb * 4 * kATile; }
__host__ __device__ constexpr int b_tile_rows(int N) { return (N + kBoxRows - 1) / kBoxRows * kBoxRows; }
__host__ __device__ constexpr int b_slot_bytes(int N) { return 2 * b_tile_rows(N) * kRowBytes; }
__host__ __device__ constexpr int smem_layout_bytes(int prec, int rb, int N)
{
    return 2 * a_buffer_bytes(rb) + 2 * aux_bytes(prec) + kBRing * b_slot_bytes(N);
}
__host__ __device__ constexpr size_t smem_max(int prec)
{
    return 1024 + (size_t)(smem_layout_bytes(prec, 2, kMaxN / 2) > smem_layout_bytes(prec, 1, kMaxN)
                               ? smem_layout_bytes(prec, 2, kMaxN / 2)
                               : smem_layout_bytes(prec, 1, kMaxN));
}
static_assert(smem_max(kPrecFP8) <= 232448 - 512, "FP8 buffers fit in shared memory");
static_assert(smem_max(kPrecBF16) <= 232448 - 512, "16-bit buffers fit in shared memory");
// epilogue staging: per producer warp 32 rows x 16 columns (pitch 17)
static_assert(kWarps * 32 * 17 * 4 <= 2 * a_buffer_bytes(1), "epilogue staging fits the A buffers");

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

// Splits two 16-bit operand values (x, y) into a 4-byte word of hi parts and
// one of lo parts, x = hi + lo up to the rounding of lo.
template <int P>
__device__ __forceinline__ void split_pair(float x, float y, uint32_t &hi, uint32_t &lo)
{
    if (P == kPrecBF16) {
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

// The split of both classes' operand values of one row and frequency, held as
// packed pairs X = (x_0, x_1), Y = (y_0, y_1): class c's pair (x_c, y_c) gives
// the words hi_c and lo_c, bit for bit as split_pair would.
template <int P>
__device__ __forceinline__ void split_classes(f32x2 X, f32x2 Y, uint32_t &h0, uint32_t &l0,
                                              uint32_t &h1, uint32_t &l1)
{
    const float2 x = unpack2(X), y = unpack2(Y);
    if (P == kPrecBF16) {
        __nv_bfloat162 a = __floats2bfloat162_rn(x.x, y.x);
        __nv_bfloat162 c = __floats2bfloat162_rn(x.y, y.y);
        const uint32_t ha = *reinterpret_cast<uint32_t *>(&a);
        const uint32_t hc = *reinterpret_cast<uint32_t *>(&c);
        // bf16 -> f32 is a shift (low half) or a mask (high half) of the bits
        const f32x2 fx = pack2(__uint_as_float(ha << 16), __uint_as_float(hc << 16));
        const f32x2 fy = pack2(__uint_as_float(ha & 0xffff0000u), __uint_as_float(hc & 0xffff0000u));
        const float2 rx = unpack2(sub2(X, fx)), ry = unpack2(sub2(Y, fy));
        __nv_bfloat162 la = __floats2bfloat162_rn(rx.x, ry.x);
        __nv_bfloat162 lc = __floats2bfloat162_rn(rx.y, ry.y);
        h0 = ha;
        h1 = hc;
        l0 = *reinterpret_cast<uint32_t *>(&la);
        l1 = *reinterpret_cast<uint32_t *>(&lc);
    } else {
        __half2 a = __floats2half2_rn(x.x, y.x);
        __half2 c = __floats2half2_rn(x.y, y.y);
        const float2 fa = __half22float2(a), fc = __half22float2(c);
        const float2 rx = unpack2(sub2(X, pack2(fa.x, fc.x)));
        const float2 ry = unpack2(sub2(Y, pack2(fa.y, fc.y)));
        __half2 la = __floats2half2_rn(rx.x, ry.x);
        __half2 lc = __floats2half2_rn(rx.y, ry.y);
        h0 = *reinterpret_cast<uint32_t *>(&a);
        h1 = *reinterpret_cast<uint32_t *>(&c);
        l0 = *reinterpret_cast<uint32_t *>(&la);
        l1 = *reinterpret_cast<uint32_t *>(&lc);
    }
}

// The same for four FP8 (e4m3) values (x, y, z, w) in one word.  Conversions
// saturate; the scaled operands stay far below e4m3's 448.
__device__ __forceinline__ void split_quad_e4m3(float x, float y, float z, float w, uint32_t &hi,
                                                uint32_t &lo)
{
    const __nv_fp8x2_storage_t h0 =
        __nv_cvt_float2_to_fp8x2(make_float2(x, y), __NV_SATFINITE, __NV_E4M3);
    const __nv_fp8x2_storage_t h1 =
        __nv_cvt_float2_to_fp8x2(make_float2(z, w), __NV_SATFINITE, __NV_E4M3);
    const float2 f0 = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(h0, __NV_E4M3)));
    const float2 f1 = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(h1, __NV_E4M3)));
    const __nv_fp8x2_storage_t l0 =
        __nv_cvt_float2_to_fp8x2(make_float2(x - f0.x, y - f0.y), __NV_SATFINITE, __NV_E4M3);
    const __nv_fp8x2_storage_t l1 =
        __nv_cvt_float2_to_fp8x2(make_float2(z - f1.x, w - f1.y), __NV_SATFINITE, __NV_E4M3);
    hi = (uint32_t)h0 | ((uint32_t)h1 << 16);
    lo = (uint32_t)l0 | ((uint32_t)l1 << 16);
}

template <int P>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t acc)
{
    if (P == kPrecFP8)
        mma_f8f6f4(d, a, b, idesc, acc);
    else
        mma_f16(d, a, b, idesc, acc);
}

// Instruction descriptor: FP32 accumulation, K-major A and B; the format
// fields are 0 = FP16 / 1 = BF16 for kind::f16 and 0 = E4M3 (both operands)
// for kind::f8f6f4.
template <int P>
__host__ __device__ constexpr uint32_t idesc_of(int N)
{
    return idesc_f16(kM, N, P == kPrecBF16);
}

// The MMA warp's stage loop for RB row blocks.  Every descriptor is a base
// descriptor whose low word (the 14-bit start-address field, shared memory
// below 256 KB, so never carrying into the rest) gets a compile-time offset
// per buffer, K-step, row block, class and hi/lo tile added, so that an MMA
// costs its issue and one 32-bit add instead of a chain of 64-bit arithmetic.
template <int P, int RB>
__device__ __forceinline__ void mma_stages(int n_stages, int lane, uint32_t tmem, uint32_t idesc,
                                           uint64_t d0, int b_off, int b_slot, int b_lo,
                                           uint64_t *full_bar, uint64_t *empty_bar,
                                           uint64_t *b_full, uint64_t *b_empty,
                                           volatile int *abort_v, int *abort_s, uint64_t wait_ns)
{
    constexpr int kAcc = kTmemCols / (2 * RB);            // columns per accumulator
    constexpr uint32_t kABuf = a_buffer_bytes(RB) >> 4;   // buffer 1's offset
    const uint32_t lo0 = (uint32_t)d0, hi0 = (uint32_t)(d0 >> 32);
    const auto desc = [hi0](uint32_t lo) { return ((uint64_t)hi0 << 32) | lo; };
    for (int s = 0; s < n_stages; ++s) {
        const int buf = s & 1, bs = s % kBRing;
        if (!*abort_v && !mbar_wait(&full_bar[buf], (uint32_t)(s >> 1) & 1u, wait_ns))
            atomicExch(abort_s, 1);
        if (!*abort_v && !mbar_wait(&b_full[bs], (uint32_t)(s / kBRing) & 1u, wait_ns))
            atomicExch(abort_s, 1);
        tc_fence_after_sync();
        if (lane == 0) {
            const uint32_t a0 = lo0 + (buf ? kABuf : 0u);
            const uint32_t bh0 = lo0 + (uint32_t)((b_off + bs * b_slot) >> 4);
            const uint32_t bl0 = bh0 + (uint32_t)(b_lo >> 4);
            const uint32_t first = s > 0 ? 1u : 0u;  // the first stage's first K-step starts the sums
#pragma unroll
            for (int kk = 0; kk < kRowBytes / 32; ++kk) {
#pragma unroll
                for (int r = 0; r < RB; ++r) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        constexpr uint32_t kT = kATile >> 4;
                        const uint32_t ah = a0 + (uint32_t)((r * 2 + c) * 2) * kT + 2u * kk;
                        const uint32_t d = tmem + (uint32_t)((2 * r + c) * kAcc);
                        mma<P>(d, desc(ah), desc(bh0 + 2u * kk), idesc, kk > 0 ? 1u : first);
                        mma<P>(d, desc(ah), desc(bl0 + 2u * kk), idesc, 1u);
                        mma<P>(d, desc(ah + kT), desc(bh0 + 2u * kk), idesc, 1u);
                    }
                }
            }
            mma_commit(&empty_bar[buf]);
            mma_commit(&b_empty[bs]);
        }
        __syncwarp();
    }
}

// One (block of cells, frequency slice) item, executed by the whole CTA: 16
// producer warps generate the A operands, one warp stages each stage's inputs,
// one copies the B operand by TMA and one issues the MMAs.  The block's columns
// lie in tile column b.tile; its rows may cross tile rows (at most
// max_block_tiles(P) of them), each row using the memories of its own tile:
// row j of the A operand is U_psi of tile (row_tile[j], b.tile).  A block has
// rb = 1 or 2 row blocks of up to 128 rows (rows j0 .. j0 + 127 and j0 + 128 ..
// j1 - 1) and N <= 256 / rb columns: the tensor memory holds rb x 2 classes
// accumulators of N columns, and the B operand (the x phasors) is shared by
// all of them.
//
// Hand-offs, all through mbarriers (no CTA-wide barrier inside the loop):
//  * the loader warp copies stage s's inputs (the memories of the block's
//    tiles, the frequencies and the row-step phasors) into the aux area of
//    buffer buf = s & 1 with per-thread async copies that land on
//    aux_full[buf]; it refills buf for stage s + 2 once every producer warp
//    has arrived on full_bar[buf] for stage s (they read the aux area before
//    arriving);
//  * the TMA warp copies stage s's B tiles (hi and lo) from the x-phasor
//    table into slot s mod 4, completing on b_full[slot]; it refills the slot
//    for stage s + 4 once the MMAs of stage s have completed (b_empty[slot]);
//  * producers wait on aux_full[buf] and, from stage 2 on, on empty_bar[buf]
//    (the tensor cores have finished reading buf), generate stage s's A
//    operands and arrive on full_bar[buf] (one arrival per warp, after a
//    proxy fence);
//  * the MMA warp waits on full_bar[buf] and b_full[slot], issues the stage's
//    MMAs and commits them to empty_bar[buf] and b_empty[slot].
// Producer warps therefore drift apart by up to a stage instead of meeting
// at a barrier every stage.  Every wait is bounded; after a time-out the CTA
// stops waiting, records VSAOGM_E_TIMEOUT, drains its MMAs and TMA copies and
// frees its tensor memory.
//
// Producer thread (warp w, lane l) owns word l mod 16 of every operand row it
// writes (frequencies FPL (l mod 16) .. + FPL - 1 of the stage, FPL = 1 for
// 16-bit operands, 2 for FP8), and the rows 8 rb w + l / 16 + 2 q, q < 4 rb:
// a warp's rows are consecutive and lie in one row block, a thread's rows
// cross into the next tile row at most once for tiles of 8 rb rows or more,
// and one store instruction of the warp fills two adjacent 64-byte rows.
// Each thread carries the two classes' operand values of a row as packed
// pairs, (Re U_0, Re U_1) and (-Im U_0, -Im U_1), so one packed multiply-add
// advances both classes.
template <int P>
__device__ __forceinline__ void decode_tc_body(
    const DecodeBlock b, const int split, const float2 *__restrict__ omega,
    const float *__restrict__ inv_norm, const float *__restrict__ nu, int D, int tiles_x,
    const int *__restrict__ row_tile, OutGeom og, const float *__restrict__ col_off,
    const float *__restrict__ row_off, const float2 *__restrict__ rot, int k_per_split,
    float u_scale, float *__restrict__ partial, int *__restrict__ status,
    uint64_t debug_wait_ns, const uint8_t *__restrict__ xtmap)
{
    constexpr int KS = stage_freqs(P);       // frequencies per stage
    constexpr int FPL = KS / kWords;         // frequencies per operand word
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[2], empty_bar[2], aux_full[2], done_bar, never_bar;
    __shared__ uint64_t b_full[kBRing], b_empty[kBRing];
    __shared__ float s_scale[2 * kMaxBlockTiles];  // 1 / norm x u_scale per (tile row, class)
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;
    volatile int *abort_v = &abort_s;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // limit of the pipeline's waits: 2 s, or the failure-test knob (the drain
    // before the tensor memory is freed always keeps the 2 s limit)
    const uint64_t wait_ns = debug_wait_ns ? debug_wait_ns : kWaitNs;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int k_begin = split * k_per_split;
    const int k_end = min(D, k_begin + k_per_split);
    const int n_stages = (k_end - k_begin + KS - 1) / KS;
    const int ni = b.i1 - b.i0, nj = b.j1 - b.j0;
    const int rb = nj > kM ? 2 : 1;               // row blocks
    const int N = (ni + 15) / 16 * 16;            // MMA N
    const int acc_cols = kTmemCols / (2 * rb);    // tensor-memory columns per accumulator
    // shared memory layout (offsets from `smem`): A buffers, aux areas, B slots
    const int a_bytes = a_buffer_bytes(rb);
    const int aux_off = 2 * a_bytes;
    const int b_off = aux_off + 2 * aux_bytes(P);
    const int b_slot = b_slot_bytes(N), b_lo = b_tile_rows(N) * kRowBytes;
    const int by0 = row_tile[b.j0];
    const int nt = row_tile[b.j1 - 1] - by0 + 1;  // tile rows of the block
    if (nt < 1 || nt > max_block_tiles(P) || ni < 1 || nj < 1 || nj > kMaxRowBlocks * kM ||
        N > kTmemCols / (2 * rb)) {
        // the host never builds such a block; refuse it rather than index past smem
        if (tid == 0) atomicExch(status, VSAOGM_E_INVAL);
        return;
    }

    if (warp == 0) {
        tmem_alloc(&tmem_base_s, kTmemCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < 2; ++q) {
            mbar_init(&full_bar[q], kWarps);
            mbar_init(&empty_bar[q], 1);
            mbar_init(&aux_full[q], 32);  // every loader lane arrives once its copies land
        }
        for (int q = 0; q < kBRing; ++q) {
            mbar_init(&b_full[q], 1);   // the TMA warp's arrival plus the copies' bytes
            mbar_init(&b_empty[q], 1);  // the MMA warp's commit
        }
        mbar_init(&done_bar, 1);
        mbar_init(&never_bar, 1);  // nothing arrives on it (failure test only)
        mbar_fence_init();
        abort_s = 0;
    }
    if (tid < 2 * nt) {
        const int mem = 2 * ((by0 + (tid >> 1)) * tiles_x + b.tile) + (tid & 1);
        s_scale[tid] = inv_norm[mem] * u_scale;
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = tmem_base_s;

    if (warp == kMmaWarp) {
        // ------------------------------------------------------ MMA warp
        // A area: tiles [row block][class][hi, lo] of 128 rows; B area: the hi
        // and the lo tile of N rows.  Descriptors are those of buffer 0; buffer
        // 1 and each K-step (32 bytes) add their byte offset / 16 to the
        // start-address field.
        const uint32_t idesc = idesc_of<P>(N);
        const uint64_t d0 = desc_k_sw64(smem_addr(smem));
        if (rb == 1)
            mma_stages<P, 1>(n_stages, lane, tmem, idesc, d0, b_off, b_slot, b_lo, full_bar,
                             empty_bar, b_full, b_empty, abort_v, &abort_s, wait_ns);
        else
            mma_stages<P, 2>(n_stages, lane, tmem, idesc, d0, b_off, b_slot, b_lo, full_bar,
                             empty_bar, b_full, b_empty, abort_v, &abort_s, wait_ns);
        // one more commit arrives when every MMA issued above has finished
        if (lane == 0) mma_commit(&done_bar);
        __syncwarp();
    } else if (warp == kLoadWarp) {
        // --------------------------------------------------- loader warp
        // aux area of a buffer: the raw memories (tile row, class, frequency)
        // as float2 [nt][2][KS], then per frequency (nu_x, nu_y) float2 [KS]
        // and the step phasors along x and y, float2 [2][KS].  Copied with
        // per-thread async copies that land on aux_full[buf]; frequencies past
        // the slice's end are zero-filled (memories 0, so their U and hence
        // their products vanish).
        const int n_w = nt * 2 * KS;
        // failure test: stall on a barrier nothing arrives at, for four times
        // the pipeline's wait limit, so that the other warps' waits run out
        if (debug_wait_ns) mbar_wait(&never_bar, 0u, 4 * debug_wait_ns);
        for (int s = 0; s < n_stages; ++s) {
            const int buf = s & 1;
            // buf's aux area held stage s - 2, which every producer has read
            // before arriving on full_bar[buf]
            if (s >= 2 && !*abort_v &&
                !mbar_wait(&full_bar[buf], (uint32_t)((s - 2) >> 1) & 1u, wait_ns))
                atomicExch(&abort_s, 1);
            float2 *aw = reinterpret_cast<float2 *>(smem + aux_off + buf * aux_bytes(P));
            float2 *af = aw + max_block_tiles(P) * 2 * KS;
            const int k0 = k_begin + s * KS;
            for (int e = lane; e < n_w; e += 32) {
                const int r = e / KS, k = k0 + e % KS;
                const int mem = 2 * ((by0 + (r >> 1)) * tiles_x + b.tile) + (r & 1);
                const bool in = k < k_end;
                cp_async<8>(&aw[e], omega + (size_t)mem * D + (in ? k : 0), in);
            }
            for (int kk = lane; kk < KS; kk += 32) {
                const int k = k0 + kk;
                const bool in = k < k_end;
                const int kc = in ? k : 0;
                cp_async<4>(&af[kk].x, nu + kc, in);
                cp_async<4>(&af[kk].y, nu + D + kc, in);
                cp_async<8>(&af[KS + kk], rot + kc, in);
                cp_async<8>(&af[2 * KS + kk], rot + D + kc, in);
            }
            cp_async_mbar_arrive(&aux_full[buf]);
        }
        cp_async_wait_all();
    } else if (warp == kBLoadWarp) {
        // ------------------------------------------------ TMA warp (B operand)
        // Slot s mod kBRing receives the x phasors (hi and lo tiles) of the
        // block's N columns and stage s's frequencies, copied from the map's
        // table by TMA boxes of 16 words x 64 rows (64-byte swizzle); rows past
        // the map read as zeros and rows past N are never used.  It refills a
        // slot once the MMAs that read it have completed (b_empty).
        if (lane == 0 && n_stages > 0) {
            const uint8_t *t_hi = xtmap, *t_lo = xtmap + 128;
            tensormap_acquire(t_hi);
            tensormap_acquire(t_lo);
            const int nbox = b_tile_rows(N) / kBoxRows;
            const uint32_t bytes = (uint32_t)(2 * nbox * kBoxRows * kRowBytes);
            for (int s = 0; s < n_stages; ++s) {
                const int bs = s % kBRing;
                if (s >= kBRing && !*abort_v &&
                    !mbar_wait(&b_empty[bs], (uint32_t)((s - kBRing) / kBRing) & 1u, wait_ns))
                    atomicExch(&abort_s, 1);
                uint8_t *dst = smem + b_off + bs * b_slot;
                const int x = (k_begin + s * KS) / FPL;  // word of the stage's first frequency
                mbar_arrive_expect_tx(&b_full[bs], bytes);
                for (int j = 0; j < nbox; ++j) {
                    tma_load_2d(dst + j * kBoxRows * kRowBytes, t_hi, x, b.i0 + j * kBoxRows,
                                &b_full[bs]);
                    tma_load_2d(dst + b_lo + j * kBoxRows * kRowBytes, t_lo, x,
                                b.i0 + j * kBoxRows, &b_full[bs]);
                }
            }
            // every copy issued has landed before the CTA may end (bounded)
            for (int s = max(0, n_stages - kBRing); s < n_stages; ++s)
                mbar_wait(&b_full[s % kBRing], (uint32_t)(s / kBRing) & 1u, kWaitNs);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------ producers
        const int wd = lane & (kWords - 1);  // word of the operand rows
        // the warp's rows: 8 rb consecutive ones from w0, all in row block
        // w0 / 128; the thread's are r0 + 2 q, q < nq
        const int w0 = 8 * rb * warp;
        const int r0 = w0 + (lane >> 4);
        const int nq = max(0, min(4 * rb, (nj - r0 + 1) / 2));  // rows inside the block
        float dy[2 * 4];
        int tl[2 * 4];  // tile row of each A row, relative to by0
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int m = r0 + kStep * q;
            const bool v = q < nq;
            dy[q] = v ? row_off[b.j0 + m] : 0.f;
            const int t = v ? row_tile[b.j0 + m] - by0 : 0;
            tl[q] = VSAOGM_IN_BOUNDS(t >= 0 && t < nt) ? t : 0;  // staged memories exist for [0, nt)
        }
        // byte of the thread's word in its row r0 + 2 q: the 64-byte swizzle
        // phase of that row, (row / 2) mod 4, is q mod 4 (w0 / 2 is a multiple of 4)
        uint32_t soff[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            soff[j] = (uint32_t)((w0 / kM) * 4 * kATile + (r0 & (kM - 1)) * kRowBytes +
                                 ((((wd >> 2) ^ j) << 4) | ((wd & 3) << 2)));
        constexpr int kQBytes = kStep * kRowBytes;  // the thread's next row
        // a warp whose rows all lie past the block writes nothing: those A
        // rows only reach accumulator rows that are never written out
        const bool gen = w0 < nj;
        uint32_t phase_bits = 0u;  // bit b: parity to wait for on empty_bar[b]

        for (int s = 0; s < n_stages; ++s) {
            const int buf = s & 1;
            if (s >= 2) {
                if (!*abort_v && !mbar_wait(&empty_bar[buf], (phase_bits >> buf) & 1u, wait_ns))
                    atomicExch(&abort_s, 1);
                phase_bits ^= 1u << buf;
            }
            if (!*abort_v && !mbar_wait(&aux_full[buf], (uint32_t)(s >> 1) & 1u, wait_ns))
                atomicExch(&abort_s, 1);
            uint8_t *st = smem + buf * a_bytes;
            if (!gen) {
                fence_async_shared();
                __syncwarp();
                if (lane == 0) mbar_arrive(&full_bar[buf]);
                continue;
            }
            const float2 *sw = reinterpret_cast<const float2 *>(smem + aux_off + buf * aux_bytes(P));
            const float2 *sf = sw + max_block_tiles(P) * 2 * KS;
            float nuy[FPL];
            float2 rsy[FPL];
#pragma unroll
            for (int j = 0; j < FPL; ++j) {
                nuy[j] = sf[FPL * wd + j].y;
                rsy[j] = sf[2 * KS + FPL * wd + j];
            }
            // No masking below: frequencies past the slice's end have staged
            // memories 0, so their U and hence their products vanish; rows and
            // columns past the block (its MMA padding) are never written out.
            //
            // (the B operand, the x phasors of the N columns, comes from the
            // map's table by TMA)
            // A operands: (Re U_psi, -Im U_psi) with U_psi = conj(w_hat_psi) x
            // the y phasor, i.e. V_psi = conj(U_psi) = w_hat_psi x conj(phasor),
            // held for both classes as packed pairs X = (Re V_0, Re V_1), Y =
            // (Im V_0, Im V_1).  Rows step by 2 cells: V times conj(exp(i 2 pi
            // nu_y 2 res)), except where a row enters the next tile: there the
            // phasor and the memories are reloaded.
            {
                f32x2 X[FPL], Y[FPL], R2[FPL], I2[FPL], NI2[FPL];
#pragma unroll
                for (int j = 0; j < FPL; ++j) {
                    R2[j] = pack2(rsy[j].x, rsy[j].x);
                    I2[j] = pack2(rsy[j].y, rsy[j].y);
                    NI2[j] = pack2(-rsy[j].y, -rsy[j].y);
                }
                auto start_row = [&](int q) {
                    const f32x2 sc = pack2(s_scale[2 * tl[q]], s_scale[2 * tl[q] + 1]);
#pragma unroll
                    for (int j = 0; j < FPL; ++j) {
                        const float2 e = phasor(nuy[j], dy[q]);
                        const float2 w0 = sw[(2 * tl[q]) * KS + FPL * wd + j];
                        const float2 w1 = sw[(2 * tl[q] + 1) * KS + FPL * wd + j];
                        // V = w_hat x conj(e), w_hat = w / norm (x u_scale)
                        X[j] = mul2(pack2(w0.x * e.x + w0.y * e.y, w1.x * e.x + w1.y * e.y), sc);
                        Y[j] = mul2(pack2(w0.y * e.x - w0.x * e.y, w1.y * e.x - w1.x * e.y), sc);
                    }
                };
                start_row(0);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (q >= nq) break;
                    if (q > 0) {
                        if (tl[q] != tl[q - 1]) {
                            start_row(q);
                        } else {
                            // V' = V x conj(r) = (a r_x + b r_y, b r_x - a r_y)
#pragma unroll
                            for (int j = 0; j < FPL; ++j) {
                                const f32x2 x = fma2(X[j], R2[j], mul2(Y[j], I2[j]));
                                Y[j] = fma2(Y[j], R2[j], mul2(X[j], NI2[j]));
                                X[j] = x;
                            }
                        }
                    }
                    // tiles [row block w0 / 128][class][hi, lo]
                    uint8_t *ra = st + q * kQBytes + soff[q & 3];
                    uint32_t h0, l0, h1, l1;
                    if (FPL == 1) {
                        split_classes<P>(X[0], Y[0], h0, l0, h1, l1);
                    } else {
                        const float2 x0 = unpack2(X[0]), y0 = unpack2(Y[0]);
                        const float2 x1 = unpack2(X[FPL - 1]), y1 = unpack2(Y[FPL - 1]);
                        split_quad_e4m3(x0.x, y0.x, x1.x, y1.x, h0, l0);
                        split_quad_e4m3(x0.y, y0.y, x1.y, y1.y, h1, l1);
                    }
                    *reinterpret_cast<uint32_t *>(ra + 0 * kATile) = h0;
                    *reinterpret_cast<uint32_t *>(ra + 1 * kATile) = l0;
                    *reinterpret_cast<uint32_t *>(ra + 2 * kATile) = h1;
                    *reinterpret_cast<uint32_t *>(ra + 3 * kATile) = l1;
                }
            }
            // hand the stage to the MMA warp
            fence_async_shared();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full_bar[buf]);
        }
    }
    // epilogue (producers): accumulator a = 2 r + c (row block r, class c)
    // holds N columns in 16-column chunks; warp w reads tensor-memory lanes
    // 32 (w mod 4) .. + 31 (its lane quarter: rows 128 r + 32 (w mod 4) + lane)
    // of every fourth chunk, starting at chunk w / 4.  Each chunk goes through
    // shared memory (free once every MMA has finished), so that each store
    // instruction writes two 64-byte row segments.  Always drain (bounded),
    // even after a time-out: tensor memory is freed below.
    if (!mbar_wait(&done_bar, 0u, kWaitNs)) atomicExch(&abort_s, 1);
    tc_fence_after_sync();
    __syncthreads();
    if (warp < kWarps && !abort_s) {
        const int lq = warp & 3, nch = N / 16;
        float *tile = reinterpret_cast<float *>(smem) + (size_t)warp * 32 * 17;
        for (int t = warp >> 2; t < 2 * rb * nch; t += 4) {
            const int a = t / nch, cc = t - a * nch, r = a >> 1, c = a & 1;
            const int row0 = r * kM + lq * 32;  // block row of lane 0 (warp-uniform)
            if (row0 >= nj) continue;
            float v[16];
            if (n_stages > 0) {
                tmem_ld_32x32b_x16(tmem + ((uint32_t)(lq * 32) << 16) +
                                       (uint32_t)(a * acc_cols + cc * 16),
                                   v);
            } else {
#pragma unroll
                for (int x = 0; x < 16; ++x) v[x] = 0.f;  // no frequencies in this slice
            }
#pragma unroll
            for (int x = 0; x < 16; ++x) tile[lane * 17 + x] = v[x];
            __syncwarp();
            float *out = partial + (((size_t)split * 2 + c) * og.OH) * og.OW;
            const int x = lane & 15, col = cc * 16 + x;
            for (int i = 0; i < 16; ++i) {
                const int rr = 2 * i + (lane >> 4), mr = row0 + rr;
                if (mr < nj && col < ni &&
                    VSAOGM_IN_BOUNDS(b.j0 + mr - og.oy >= 0 && b.j0 + mr - og.oy < og.OH &&
                                     b.i0 + col - og.ox >= 0 && b.i0 + col - og.ox < og.OW))
                    out[(size_t)(b.j0 + mr - og.oy) * og.OW + (b.i0 + col - og.ox)] =
                        tile[rr * 17 + x];
            }
            __syncwarp();
        }
    }
    if (abort_s && tid == 0) atomicExch(status, VSAOGM_E_TIMEOUT);
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

template <int P>
__global__ void __launch_bounds__(kThreads, 1) decode_tc_kernel(
    const BlockBatch blocks, const float2 *__restrict__ omega, const float *__restrict__ inv_norm,
    const float *__restrict__ nu, int D, int tiles_x, const int *__restrict__ row_tile, OutGeom og,
    const float *__restrict__ col_off, const float *__restrict__ row_off,
    const float2 *__restrict__ rot, int k_per_split, float u_scale,
    float *__restrict__ partial, int *__restrict__ status, uint64_t debug_wait_ns,
    const uint8_t *__restrict__ xtmap)
{
    decode_tc_body<P>(blocks.b[blockIdx.x], blockIdx.y, omega, inv_norm, nu, D, tiles_x, row_tile,
                      og, col_off, row_off, rot, k_per_split, u_scale, partial, status,
                      debug_wait_ns, xtmap);
}

// Many maps in one launch: CTA q decodes item q of a device list of
// (map, block, slice); each map's pointers come from the table.
template <int P>
__global__ void __launch_bounds__(kThreads, 1) decode_tc_batch_kernel(
    const __grid_constant__ BatchDecodeTable tab, const BatchDecodeItem *__restrict__ items)
{
    const BatchDecodeItem it = items[blockIdx.x];
    const BatchDecodeMap &M = tab.m[it.map];
    decode_tc_body<P>(it.b, it.split, M.omega, M.inv_norm, M.nu, M.D, M.tiles_x, M.row_tile,
                      OutGeom{0, 0, M.W, M.H}, M.col_off, M.row_off, M.rot, M.k_per_split,
                      M.u_scale, M.partial, M.status, M.debug_wait_ns, M.xtmap);
}

// rot[k] = exp(i 2 pi nu[k] step) for the x frequencies, then the y ones: the
// phasor of one step between a producer thread's rows (kStep cells).  The phase is
// reduced exactly and sin / cos taken of the reduced turn (sincospi).
__global__ void __launch_bounds__(256) tc_rot_kernel(const float *__restrict__ nu, int n,
                                                     float step, float2 *__restrict__ rot)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float kMagic = 12582912.0f;
    const float v = nu[k];
    float p = __fmul_rn(v, step);
    float e = fmaf(v, step, -p);
    float r = __fsub_rn(__fadd_rn(p, kMagic), kMagic);
    float f = __fadd_rn(__fsub_rn(p, r), e);
    float sn, cs;
    sincospif(2.f * f, &sn, &cs);
    rot[k] = make_float2(cs, sn);
}

// The x-phasor table of the B operand: plane 0 the hi parts, plane 1 the lo
// parts, each [W columns][Dp words] with word w of column c holding the split
// x phasor(s) exp(i 2 pi nu_x[k] dx_c) of frequency k = w (16-bit formats) or
// k = 2w, 2w + 1 (FP8) in the layout of one operand row; words past D are 0.
// Built once per map: it depends only on the frequencies and the geometry.
template <int P>
__global__ void __launch_bounds__(256) tc_xtab_kernel(const float *__restrict__ nu,
                                                      const float *__restrict__ col_off, int D,
                                                      int W, int Dp, uint32_t *__restrict__ tab)
{
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= (size_t)W * Dp) return;
    constexpr int FW = P == kPrecFP8 ? 2 : 1;  // frequencies per word
    const int c = (int)(i / Dp), w = (int)(i % Dp);
    float2 v[FW];
#pragma unroll
    for (int j = 0; j < FW; ++j) {
        const int k = FW * w + j;
        v[j] = k < D ? phasor(nu[k], col_off[c]) : make_float2(0.f, 0.f);
    }
    uint32_t hi, lo;
    if (FW == 1)
        split_pair<P>(v[0].x, v[0].y, hi, lo);
    else
        split_quad_e4m3(v[0].x, v[0].y, v[FW - 1].x, v[FW - 1].y, hi, lo);
    tab[i] = hi;
    tab[(size_t)W * Dp + i] = lo;
}

int prec_of(int decode_prec)
{
    return decode_prec == VSAOGM_DECODE_FP8X3   ? kPrecFP8
           : decode_prec == VSAOGM_DECODE_FP16X3 ? kPrecFP16
                                                 : kPrecBF16;
}

template <int P>
cudaError_t set_smem_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(decode_tc_kernel<P>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_max(P));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(decode_tc_batch_kernel<P>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max(P));
    return e;
}

}  // namespace

int tc_stage_freqs(int decode_prec) { return stage_freqs(prec_of(decode_prec)); }

VSAOGM_CHECK_TU(decode_tc)

// Blocks covering region r for the tensor-core decode, one CTA each: columns
// inside one tile column, rows across at most max_block_tiles tile rows.  In
// a tile column wider than 128 cells a block is one row block (up to 128 rows)
// by up to 256 columns, the column range cut into equal parts; in a narrower
// one it is two row blocks (up to 256 rows) by the whole tile column, so the
// x-phasor operand serves twice the rows.  Either way the tensor memory holds
// the block's accumulators (row blocks x 2 classes x N <= 512 columns).
void tc_blocks(const vsaogm_map *m, Region r, std::vector<DecodeBlock> &out)
{
    out.clear();
    const int max_tiles = max_block_tiles(prec_of(m->cfg.decode_prec));
    const std::vector<int> &yl = m->tile_last[1];  // tiles are monotonic in the row index
    const int ty = m->cfg.tiles_y;
    for (int bx = 0; bx < m->cfg.tiles_x; ++bx) {
        const int x0 = std::max(r.x0, m->tile_first[0][bx]);
        const int x1 = std::min(r.x1, m->tile_last[0][bx]);
        const int w = x1 - x0;
        if (w <= 0) continue;
        const bool wide = w > kM;
        const int parts = wide ? (w + kMaxN - 1) / kMaxN : 1;
        const int rows_max = wide ? kM : kMaxRowBlocks * kM;
        for (int p = 0; p < parts; ++p) {
            const int i0 = x0 + (int)((long long)w * p / parts);
            const int i1 = x0 + (int)((long long)w * (p + 1) / parts);
            int by = 0;
            for (int j0 = r.y0; j0 < r.y1;) {
                while (by < ty - 1 && yl[by] <= j0) ++by;  // tile row of row j0
                // rows up to the end of the max_tiles-th tile row from by
                int cap = j0 + 1;
                for (int t = by; t < std::min(by + max_tiles, ty); ++t) cap = std::max(cap, yl[t]);
                const int j1 = std::min({j0 + rows_max, r.y1, cap});
                out.push_back(DecodeBlock{bx, i0, j0, i1, j1});
                j0 = j1;
            }
        }
    }
}

int launch_decode_tc_batch(const BatchDecodeTable &tab, const BatchDecodeItem *items,
                           int n_items, int decode_prec, cudaStream_t st)
{
    const int P = prec_of(decode_prec);
    cudaError_t e = P == kPrecFP8    ? set_smem_attributes<kPrecFP8>()
                    : P == kPrecFP16 ? set_smem_attributes<kPrecFP16>()
                                     : set_smem_attributes<kPrecBF16>();
    if (e == cudaSuccess) {
        const size_t smem = smem_max(P);
        if (P == kPrecFP8)
            decode_tc_batch_kernel<kPrecFP8><<<n_items, kThreads, smem, st>>>(tab, items);
        else if (P == kPrecFP16)
            decode_tc_batch_kernel<kPrecFP16><<<n_items, kThreads, smem, st>>>(tab, items);
        else
            decode_tc_batch_kernel<kPrecBF16><<<n_items, kThreads, smem, st>>>(tab, items);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? VSAOGM_OK : cuda_error(e, "batch decode");
}

// Power-of-two scale of U for the FP16 and FP8 operands (U = conj(w_hat) x
// phasor has |U_k| ~ 1 / sqrt(D)): u with 4 u^2 <= D, undone by the slice sum.
float tc_u_scale(const vsaogm_map *m)
{
    float u = 1.f;
    if (m->cfg.decode_prec == VSAOGM_DECODE_FP16X3 || m->cfg.decode_prec == VSAOGM_DECODE_FP8X3)
        while (u * u * 4.f <= (float)m->cfg.D) u *= 2.f;
    return u;
}

int build_tc_tables(vsaogm_map *m)
{
    const int D = m->cfg.D;
    cudaError_t e = dev_malloc((void **)&m->tc_rot, sizeof(float2) * 2 * (size_t)D);
    if (e != cudaSuccess) return cuda_error(e, "decode tables");
    // the same float step as the kernel's rows and columns: kStep cells
    tc_rot_kernel<<<(2 * D + 255) / 256, 256>>>(m->nu, 2 * D, (float)kStep * m->cfg.resolution,
                                                m->tc_rot);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "decode tables");
    // the x-phasor table of the B operand and its two TMA tensor maps
    const int P = prec_of(m->cfg.decode_prec);
    const int W = m->cfg.grid_w;
    const int words = P == kPrecFP8 ? (D + 1) / 2 : D;
    const int Dp = (words + kWords - 1) / kWords * kWords;  // whole 64-byte boxes
    const size_t plane = (size_t)W * Dp;
    if ((e = dev_malloc((void **)&m->tc_xtab, sizeof(uint32_t) * 2 * plane)) != cudaSuccess)
        return cuda_error(e, "decode tables");
    const unsigned grid = (unsigned)((plane + 255) / 256);
    if (P == kPrecFP8)
        tc_xtab_kernel<kPrecFP8><<<grid, 256>>>(m->nu, m->col_off, D, W, Dp, m->tc_xtab);
    else if (P == kPrecFP16)
        tc_xtab_kernel<kPrecFP16><<<grid, 256>>>(m->nu, m->col_off, D, W, Dp, m->tc_xtab);
    else
        tc_xtab_kernel<kPrecBF16><<<grid, 256>>>(m->nu, m->col_off, D, W, Dp, m->tc_xtab);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess)
        return cuda_error(e, "decode tables");
    PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    cudaDriverEntryPointQueryResult q;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void **)&encode, 12000,
                                         cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !encode)
        return set_error(VSAOGM_E_CUDA, "decode tables: cuTensorMapEncodeTiled unavailable");
    CUtensorMap maps[2];
    for (int h = 0; h < 2; ++h) {
        // [W rows][Dp words] of 4 bytes; a box is one 64-byte operand row
        // (16 words) by kBoxRows columns, written with the 64-byte swizzle
        const cuuint64_t dims[2] = {(cuuint64_t)Dp, (cuuint64_t)W};
        const cuuint64_t strides[1] = {(cuuint64_t)Dp * 4};
        const cuuint32_t box[2] = {(cuuint32_t)kWords, (cuuint32_t)kBoxRows};
        const cuuint32_t elem[2] = {1, 1};
        CUresult r = encode(&maps[h], CU_TENSOR_MAP_DATA_TYPE_UINT32, 2,
                            (void *)(m->tc_xtab + h * plane), dims, strides, box, elem,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return set_error(VSAOGM_E_CUDA, "decode tables: tensor map (error %d)", (int)r);
    }
    if ((e = dev_malloc((void **)&m->tc_xtmap, sizeof(maps))) != cudaSuccess)
        return cuda_error(e, "decode tables");
    if ((e = cudaMemcpy(m->tc_xtmap, maps, sizeof(maps), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_error(e, "decode tables");
    return VSAOGM_OK;
}

int decode_tensor_cores(vsaogm_map *m, Region r, float *heat, cudaStream_t st)
{
    const int D = m->cfg.D;
    const int P = prec_of(m->cfg.decode_prec);
    const int KS = stage_freqs(P);
    std::vector<DecodeBlock> blocks;
    tc_blocks(m, r, blocks);
    const int nb = (int)blocks.size();
    // slices of the frequencies so that blocks x slices fills the 152 SMs once,
    // and no slice longer than kTcMaxKPerSplit
    int splits = std::max((D + kTcMaxKPerSplit - 1) / kTcMaxKPerSplit,
                          std::min((D + KS - 1) / KS, 152 / std::max(nb, 1)));
    int kps = ((D + splits - 1) / splits + KS - 1) / KS * KS;
    splits = (D + kps - 1) / kps;
    const size_t cells = (size_t)r.w() * r.h();
    int rc = ensure(m->ws.dec_partial, sizeof(float) * (size_t)splits * 2 * cells);
    if (rc) return rc;
    const float u_scale = tc_u_scale(m);
    cudaError_t e = P == kPrecFP8    ? set_smem_attributes<kPrecFP8>()
                    : P == kPrecFP16 ? set_smem_attributes<kPrecFP16>()
                                     : set_smem_attributes<kPrecBF16>();
    if (e != cudaSuccess) return cuda_error(e, "decode: tensor cores");
    StageScope sc(m, VSAOGM_STAGE_DECODE, st);
    float *part = (float *)m->ws.dec_partial.ptr;
    const OutGeom og{r.x0, r.y0, r.w(), r.h()};
    int launches = 0;
    for (int b0 = 0; b0 < nb; b0 += kMaxLaunchBlocks) {
        BlockBatch batch;
        batch.n = std::min(kMaxLaunchBlocks, nb - b0);
        for (int q = 0; q < batch.n; ++q) batch.b[q] = blocks[b0 + q];
        const size_t smem = smem_max(P);
        dim3 grid(batch.n, splits);
#define VSAOGM_LAUNCH_TC(PP)                                                                   \
    decode_tc_kernel<PP><<<grid, kThreads, smem, st>>>(                                        \
        batch, m->omega, m->inv_norm, m->nu, D, m->cfg.tiles_x, m->row_tile, og, m->col_off,    \
        m->row_off, m->tc_rot, kps, u_scale, part, m->status, m->debug_wait_ns, m->tc_xtmap)
        if (P == kPrecFP8)
            VSAOGM_LAUNCH_TC(kPrecFP8);
        else if (P == kPrecFP16)
            VSAOGM_LAUNCH_TC(kPrecFP16);
        else
            VSAOGM_LAUNCH_TC(kPrecBF16);
#undef VSAOGM_LAUNCH_TC
        ++launches;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "decode: tensor cores");
    if ((rc = sum_slices(m, part, splits, cells, 1.0f / u_scale, heat, st))) return rc;
    sc.end(launches + 1);
    return VSAOGM_OK;
}

}  // namespace vsaogm_impl
