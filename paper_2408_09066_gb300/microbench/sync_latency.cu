// Hand-off latency microbenchmark for the decode pipeline's synchronisation
// steps on one SM: an mbarrier round trip between two warps (plain test loop
// and the suspend-hint wait the kernels use), a tcgen05.commit round trip
// with no MMA and with one 128 x 128 x 16 MMA outstanding, and a warp's
// tensor-memory stores (4 x 32x32b.x8) followed by tcgen05.wait::st.  Each
// figure is clocks per iteration over many iterations (clock64), one CTA per
// SM on every SM.
//
// Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -I../csrc -o sync_latency sync_latency.cu && ./sync_latency
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

constexpr int kIters = 4096;
constexpr uint64_t kLimit = 1000000000ull;  // 1 s per wait: far above any real latency

// plain test loop, bounded by an iteration count
__device__ __forceinline__ bool spin_wait(uint64_t *bar, uint32_t parity)
{
    for (uint32_t i = 0; i < (1u << 28); ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// test: 0 ping-pong (spin), 1 ping-pong (suspend-hint wait), 2 commit without
// MMA, 3 commit after one MMA, 4 tensor-memory stores + wait::st (per warp)
__global__ void __launch_bounds__(640, 1) sync_kernel(int test, unsigned long long *out, int *err)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar_a, bar_b, bar_c;
    __shared__ volatile int busy_done;
    __shared__ uint32_t tmem_s;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < 16384 / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) {
        tmem_alloc(&tmem_s, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&bar_a, 1);
        mbar_init(&bar_b, 1);
        mbar_init(&bar_c, 1);
        busy_done = 0;
        mbar_fence_init();
    }
    fence_async_shared();
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = tmem_s;
    unsigned long long t0 = 0, t1 = 0;
    bool ok = true;
    if (test <= 1) {
        if (warp == 0 || warp == 1) {
            t0 = clock64();
            for (int i = 0; i < kIters; ++i) {
                const uint32_t par = (uint32_t)i & 1u;
                if (warp == 0) {
                    if (lane == 0) mbar_arrive(&bar_a);
                    ok &= test == 0 ? spin_wait(&bar_b, par) : mbar_wait(&bar_b, par, kLimit);
                } else {
                    ok &= test == 0 ? spin_wait(&bar_a, par) : mbar_wait(&bar_a, par, kLimit);
                    if (lane == 0) mbar_arrive(&bar_b);
                }
            }
            t1 = clock64();
        }
    } else if (test <= 3) {
        if (warp == 0) {
            const uint64_t da = desc_k_sw64(smem_addr(smem)), db = desc_k_sw64(smem_addr(smem + 8192));
            const uint32_t idesc = idesc_f16(128, 128, true);
            t0 = clock64();
            for (int i = 0; i < kIters; ++i) {
                if (lane == 0) {
                    if (test == 3) mma_f16(tmem, da, db, idesc, 1u);
                    mma_commit(&bar_a);
                }
                __syncwarp();
                ok &= mbar_wait(&bar_a, (uint32_t)i & 1u, kLimit);
            }
            t1 = clock64();
        }
    } else if (test >= 5 && warp >= 4) {
        // tests 9, 10: 16 more warps keep the schedulers busy (dependent FMA
        // chains, or MUFU sin / cos) until the MMA loop ends (bounded)
        // test 11: FMA chains only in warps of the other three schedulers
        // (warp w runs on sub-partition w mod 4; the MMA loop is warp 0's)
        if (test >= 9 && !(test == 11 && (warp & 3) == 0)) {
            float a = (float)tid * 1e-3f, b2 = a + 0.5f, c2 = a + 0.25f, d2 = a + 0.75f;
            for (int i = 0; i < (1 << 22) && !busy_done; ++i) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    if (test != 10) {
                        a = fmaf(a, 0.999f, 0.001f);
                        b2 = fmaf(b2, 0.999f, 0.001f);
                        c2 = fmaf(c2, 0.999f, 0.001f);
                        d2 = fmaf(d2, 0.999f, 0.001f);
                    } else {
                        a = __sinf(a) + b2;
                        b2 = __cosf(b2) + c2;
                    }
                }
            }
            if (a == 12345.f && b2 == 1.f && c2 == 2.f && d2 == 3.f) atomicExch(err, 2);
        }
    } else if (test >= 5) {
        // the decode's MMA-warp loop shape on completed barriers: per stage 4
        // x (test of a completed barrier, fence, 6 MMAs N = 64 with A in tensor
        // memory), then 2 commits; 5: all of it, 6: no barrier tests, 7: no
        // fences, 8: a completed-barrier test alone (per iteration)
        if (warp == 0 && lane == 0) {
            mbar_arrive(&bar_b);  // phase 0 of bar_b completes: parity-0 tests pass at once
            const uint64_t db = desc_k_sw128(smem_addr(smem));
            const uint32_t idesc = idesc_f16(128, 64, true);
            t0 = clock64();
            for (int i = 0; i < kIters / 8; ++i) {
                if (test == 8) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) ok &= mbar_try_wait(&bar_b, 0u);
                    continue;
                }
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    if (test != 6) ok &= mbar_try_wait(&bar_b, 0u);
                    if (test != 7) tc_fence_after_sync();
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const uint32_t ah = 256u + (uint32_t)(64 * c + 8 * kk);
                        mma_f16_ta((uint32_t)(c * 64), ah, db + (uint64_t)(2 * kk), idesc, 1u);
                        mma_f16_ta((uint32_t)(c * 64), ah, db + (uint64_t)(2 * kk + 1024), idesc, 1u);
                        mma_f16_ta((uint32_t)(c * 64), ah + 32u, db + (uint64_t)(2 * kk), idesc, 1u);
                    }
                }
                mma_commit(&bar_a);
            }
            t1 = clock64();
            // drain: one more commit on a fresh barrier arrives once every MMA is done
            mma_commit(&bar_c);
            ok &= mbar_wait(&bar_c, 0u, kLimit);
            t1 = (t1 - t0) * 8 / (test == 8 ? 8 : 1);
            t0 = 0;
            busy_done = 1;
        }
        __syncwarp();
    } else {
        uint32_t v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + 256u;
        t0 = clock64();
        for (int i = 0; i < kIters; ++i) {
            v[0] = (uint32_t)i;
            tmem_st_32x32b_x8(ta + 0, v);
            tmem_st_32x32b_x8(ta + 32, v);
            tmem_st_32x32b_x8(ta + 64, v);
            tmem_st_32x32b_x8(ta + 96, v);
            tmem_wait_st();
        }
        t1 = clock64();
    }
    if (!ok) atomicExch(err, 1);
    if (tid == 0) out[blockIdx.x] = t1 - t0;
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

int main()
{
    cudaDeviceProp p;
    CK(cudaGetDeviceProperties(&p, 0));
    const int sms = p.multiProcessorCount;
    const int smem = 120 * 1024;  // one CTA per SM (each allocates the whole tensor memory)
    CK(cudaFuncSetAttribute(sync_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    unsigned long long *out;
    int *err;
    CK(cudaMalloc(&out, sizeof(unsigned long long) * sms));
    CK(cudaMalloc(&err, sizeof(int)));
    unsigned long long *h = new unsigned long long[sms];
    const char *names[] = {"mbarrier round trip, spin", "mbarrier round trip, suspend-hint wait",
                           "tcgen05.commit round trip, no MMA",
                           "tcgen05.commit round trip, one 128x128x16 MMA",
                           "4 x tcgen05.st 32x32b.x8 + wait::st",
                           "stage: 4 x (test, fence, 6 MMA) + commit",
                           "stage without barrier tests",
                           "stage without fences",
                           "one test of a completed barrier",
                           "stage, 16 warps of FMA chains beside",
                           "stage, 16 warps of MUFU sin/cos beside",
                           "stage, 12 FMA warps on the other schedulers"};
    for (int test = 0; test < 12; ++test) {
        CK(cudaMemset(err, 0, sizeof(int)));
        double best = 1e30;
        for (int rep = 0; rep < 3; ++rep) {
            sync_kernel<<<sms, test >= 9 ? 640 : 128, smem>>>(test, out, err);
            CK(cudaGetLastError());
            CK(cudaDeviceSynchronize());
            CK(cudaMemcpy(h, out, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost));
            double mean = 0;
            for (int i = 0; i < sms; ++i) mean += (double)h[i];
            mean /= sms;
            best = mean < best ? mean : best;
        }
        int herr = 0;
        CK(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
        printf("%-48s %8.1f clk per iteration%s\n", names[test], best / kIters,
               herr ? "  (a wait timed out)" : "");
    }
    delete[] h;
    return 0;
}
