// Tensor-core issue-rate microbenchmark for the decode's MMA shapes: single-CTA
// tcgen05.mma (kind::f16 BF16 and kind::f8f6f4 E4M3, M = 128, FP32
// accumulation) with K-major operands in shared memory (64- or 128-byte
// swizzle) or the A operand in tensor memory, optionally while 16 other warps
// store to shared memory at full rate (as the decode's operand producers do).
// The rates bound what a decode CTA can reach: flops per SM and clock for one
// MMA shape, and how much the tensor pipe slows when shared memory also serves
// ordinary stores.
//
// One CTA per SM; warp 0 lane 0 issues `iters` x (K-steps per operand row)
// MMAs back to back into `naccs` accumulators in turn, commits them to an
// mbarrier and waits (bounded); clock64 around the loop gives clocks per MMA.
// Store warps, when enabled, write 16 bytes per lane per iteration to a
// region the MMAs never read, until the issuing thread raises a flag (or
// after a fixed iteration limit).  Operand contents are zeros.
//
// Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -I../csrc -o mma_rates mma_rates.cu && ./mma_rates
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#include "sm100.cuh"

using namespace vsaogm_impl::sm100;

#define CK(x)                                                                           \
    do {                                                                                \
        cudaError_t e_ = (x);                                                           \
        if (e_ != cudaSuccess) {                                                        \
            printf("CUDA %s @%d\n", cudaGetErrorString(e_), __LINE__);                 \
            return 1;                                                                   \
        }                                                                               \
    } while (0)

struct Cfg {
    int N;       // MMA N (16 .. 256, multiple of 16)
    int sw;      // 64 or 128: operand row bytes and swizzle
    int a_tmem;  // A operand in tensor memory (BF16 only)
    int fp8;     // kind::f8f6f4 E4M3 (K = 32) instead of kind::f16 BF16 (K = 16)
    int stores;  // 16 warps store to shared memory meanwhile
    int naccs;   // accumulators cycled through (N x naccs <= 256 with A in TMEM, else 512)
};

constexpr int kThreads = 128 + 512;
constexpr int kABytes = 128 * 128;          // A tile: 128 rows x up to 128 bytes
constexpr int kBBytes = 256 * 128;          // B tile: up to 256 rows x 128 bytes
constexpr int kStoreBytes = 16 * 32 * 16 * 8;  // 16 warps x 32 lanes x 16 B x 8 slots
constexpr int kSmem = 1024 + kABytes + kBBytes + kStoreBytes;
constexpr int kSmemRequest = 160 * 1024;    // forces one CTA per SM
static_assert(kSmem <= kSmemRequest, "layout fits the request");

__device__ __forceinline__ void mma_f16_a_tmem(uint32_t d, uint32_t a_tmem, uint64_t b,
                                               uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tmem_st_zero_x8(uint32_t taddr)
{
    const uint32_t z = 0u;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
        "r"(z)
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(kThreads, 1)
    mma_rate_kernel(Cfg c, int iters, unsigned long long *clk, unsigned long long *stored, int *err)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_s;
    __shared__ volatile int done;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *A = smem, *B = smem + kABytes, *S = smem + kABytes + kBBytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < (kABytes + kBBytes) / 16; i += kThreads)
        reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) {
        tmem_alloc(&tmem_s, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        done = 0;
    }
    fence_async_shared();
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = tmem_s;
    if (c.a_tmem && warp < 4) {
        // columns 256 .. 256 + 31 of this warp's lane quarter hold A (zeros)
        for (int col = 0; col < 32; col += 8)
            tmem_st_zero_x8(tmem + ((uint32_t)(warp * 32) << 16) + 256u + (uint32_t)col);
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();

    const int ksteps = c.sw / 32;  // 32-byte K-steps per operand row
    if (warp == 0) {
        if (lane == 0) {
            const uint32_t idesc = idesc_f16(128, c.N, !c.fp8);
            const uint64_t da = c.sw == 128 ? desc_k_sw128(smem_addr(A)) : desc_k_sw64(smem_addr(A));
            const uint64_t db = c.sw == 128 ? desc_k_sw128(smem_addr(B)) : desc_k_sw64(smem_addr(B));
            // descriptors and addresses of one group of 8 MMAs, computed once
            uint64_t a8[8], b8[8];
            uint32_t d8[8], t8[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int kk = j % ksteps;
                a8[j] = da + (uint64_t)(kk * 2);
                b8[j] = db + (uint64_t)(kk * 2);
                t8[j] = tmem + 256u + (uint32_t)(kk * 8);
                d8[j] = tmem + (uint32_t)((j % c.naccs) * c.N);
            }
            const int groups = iters * ksteps / 8;
            const unsigned long long t0 = clock64();
            if (c.a_tmem) {
                for (int g = 0; g < groups; ++g) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) mma_f16_a_tmem(d8[j], t8[j], b8[j], idesc, 1u);
                }
            } else if (c.fp8) {
                for (int g = 0; g < groups; ++g) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) mma_f8f6f4(d8[j], a8[j], b8[j], idesc, 1u);
                }
            } else {
                for (int g = 0; g < groups; ++g) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) mma_f16(d8[j], a8[j], b8[j], idesc, 1u);
                }
            }
            const unsigned long long t_issued = clock64();
            mma_commit(&bar);
            const bool ok = mbar_wait(&bar, 0u, 2000000000ull);
            const unsigned long long t1 = clock64();
            if (!ok) atomicExch(err, 1);
            clk[blockIdx.x] = t1 - t0;
            clk[gridDim.x + blockIdx.x] = t_issued - t0;
            done = 1;
        }
        __syncwarp();
    } else if (warp >= 4 && c.stores) {
        // 16 B per lane per iteration, 8 slots per lane, never read by the MMAs
        // slot j of a warp: 512 contiguous bytes, lane l at byte 16 l (no bank conflicts)
        const uint32_t base = smem_addr(S + (warp - 4) * 8 * 512 + lane * 16);
        unsigned long long n = 0;
        const uint32_t v = (uint32_t)tid;
        while (!done && n < (1ull << 26)) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" ::"r"(base + 512u * j),
                             "r"(v)
                             : "memory");
            n += 8;
        }
        atomicAdd(stored, n * 16ull);
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

int main()
{
    cudaDeviceProp p;
    CK(cudaGetDeviceProperties(&p, 0));
    const int sms = p.multiProcessorCount;
    printf("name=%s sms=%d cc=%d.%d\n", p.name, sms, p.major, p.minor);
    CK(cudaFuncSetAttribute(mma_rate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            kSmemRequest));
    unsigned long long *clk, *stored;
    int *err;
    CK(cudaMalloc(&clk, sizeof(unsigned long long) * 2 * sms));
    CK(cudaMalloc(&stored, sizeof(unsigned long long)));
    CK(cudaMalloc(&err, sizeof(int)));
    const Cfg cfgs[] = {
        // N, sw, a_tmem, fp8, stores, naccs
        {128, 64, 0, 0, 0, 1}, {128, 64, 0, 0, 0, 4}, {256, 64, 0, 0, 0, 1}, {256, 64, 0, 0, 0, 2},
        {128, 128, 0, 0, 0, 1}, {256, 128, 0, 0, 0, 1},
        {128, 64, 1, 0, 0, 1}, {128, 64, 1, 0, 0, 2}, {256, 64, 1, 0, 0, 1},
        {128, 64, 0, 1, 0, 1}, {256, 64, 0, 1, 0, 1},
        {128, 64, 0, 0, 1, 4}, {256, 64, 0, 0, 1, 2}, {128, 64, 1, 0, 1, 2}, {256, 64, 1, 0, 1, 1},
        {64, 64, 0, 0, 0, 1}, {64, 64, 1, 0, 0, 1}, {192, 64, 1, 0, 0, 1}, {128, 128, 0, 0, 1, 1},
    };
    unsigned long long *h = new unsigned long long[2 * sms];
    for (const Cfg &c : cfgs) {
        const int mmas = 24576;
        const int iters = mmas / (c.sw / 32);
        double best = 1e30, issued = 0;
        unsigned long long st = 0;
        for (int rep = 0; rep < 3; ++rep) {
            CK(cudaMemset(stored, 0, sizeof(unsigned long long)));
            CK(cudaMemset(err, 0, sizeof(int)));
            mma_rate_kernel<<<sms, kThreads, kSmemRequest>>>(c, iters, clk, stored, err);
            CK(cudaGetLastError());
            CK(cudaDeviceSynchronize());
            int herr = 0;
            CK(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
            if (herr) {
                printf("wait timed out\n");
                return 1;
            }
            CK(cudaMemcpy(h, clk, sizeof(unsigned long long) * 2 * sms, cudaMemcpyDeviceToHost));
            unsigned long long s = 0;
            CK(cudaMemcpy(&s, stored, sizeof(s), cudaMemcpyDeviceToHost));
            double mean = 0, mi = 0;
            for (int i = 0; i < sms; ++i) {
                mean += (double)h[i];
                mi += (double)h[sms + i];
            }
            mean /= sms;
            mi /= sms;
            if (mean < best) {
                best = mean;
                issued = mi;
                st = s;
            }
        }
        const int K = c.fp8 ? 32 : 16;
        const double cpm = best / mmas;  // clocks per MMA
        const double fpc = 2.0 * 128 * c.N * K / cpm;
        const double smem_rd = (c.a_tmem ? 0.0 : 128.0 * 32) + c.N * 32.0;  // MMA operand bytes
        printf("N=%3d sw=%3d A=%s %s stores=%d accs=%d: %.1f clk/MMA  %.0f flop/clk/SM  "
               "operand reads %.1f B/clk  stores %.1f B/clk  (issue loop ends at %.0f%%)\n",
               c.N, c.sw, c.a_tmem ? "tmem" : "smem", c.fp8 ? "e4m3" : "bf16", c.stores, c.naccs,
               cpm, fpc, smem_rd / cpm, (double)st / sms / best, 100.0 * issued / best);
    }
    delete[] h;
    return 0;
}
