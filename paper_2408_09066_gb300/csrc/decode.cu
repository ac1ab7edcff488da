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
__global__ void __launch_bounds__(256) norms_kernel(const float2 *__restrict__ omega, int D,
                                                    float *__restrict__ inv_norm)
{
    const int s = blockIdx.x;
    float acc = 0.f;
    for (int k = threadIdx.x; k < D; k += blockDim.x) {
        float2 w = omega[(size_t)s * D + k];
        acc = fmaf(w.x, w.x, fmaf(w.y, w.y, acc));
    }
    __shared__ float red[8];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        inv_norm[s] = t > 0.f ? rsqrtf(t) : 0.f;
    }
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

__global__ void __launch_bounds__(256) decode_fp32_kernel(
    const DecodeBlock *__restrict__ blocks, const float2 *__restrict__ omega,
    const float *__restrict__ inv_norm, const float *__restrict__ nu, int D, int W, int H,
    const float *__restrict__ col_off, const float *__restrict__ row_off,
    float *__restrict__ heat, unsigned *__restrict__ maxima)
{
    __shared__ float2 sA[kKC][kBI];
    __shared__ float2 sU[2][kKC][kBJ];
    const DecodeBlock b = blocks[blockIdx.x];
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

    for (int k0 = 0; k0 < D; k0 += kKC) {
        // tables for this stage: 2048 A entries and 2048 B entries (x2 classes)
        for (int e = threadIdx.x; e < kKC * kBI; e += blockDim.x) {
            int kk = e / kBI, ii = e % kBI;
            int k = k0 + kk, i = b.i0 + ii;
            float2 a = make_float2(0.f, 0.f);
            if (k < D && i < b.i1) a = unit_phasor(nu[k], col_off[i]);
            sA[kk][ii] = a;
        }
        for (int e = threadIdx.x; e < kKC * kBJ; e += blockDim.x) {
            int kk = e / kBJ, jj = e % kBJ;
            int k = k0 + kk, j = b.j0 + jj;
            float2 u0 = make_float2(0.f, 0.f), u1 = u0;
            if (k < D && j < b.j1) {
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
    // epilogue: store and fold the per-class maximum
    float mx[2] = {-INFINITY, -INFINITY};
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        int j = b.j0 + ty + 16 * v;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int i = b.i0 + tx + 16 * q;
            if (i < b.i1 && j < b.j1) {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    heat[((size_t)c * H + j) * W + i] = acc[c][v][q];
                    mx[c] = fmaxf(mx[c], acc[c][v][q]);
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        float m = mx[c];
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0 && m > -INFINITY) atomicMax(&maxima[c], float_to_ordered(m));
    }
}

// P -> P_hat = (P / m)^2, or 0 where the class maximum m is not positive.
__global__ void nonlinear_kernel(float *__restrict__ heat, size_t cells,
                                 const unsigned *__restrict__ maxima)
{
    const float m0 = ordered_to_float(maxima[0]), m1 = ordered_to_float(maxima[1]);
    const float i0 = m0 > 0.f ? 1.0f / m0 : 0.f, i1 = m1 > 0.f ? 1.0f / m1 : 0.f;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < 2 * cells;
         q += (size_t)gridDim.x * blockDim.x) {
        float v = heat[q] * (q < cells ? i0 : i1);
        heat[q] = v * v;
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
    norms_kernel<<<m->S, 256, 0, st>>>(m->omega, m->cfg.D, m->inv_norm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "decode: norms");
    sc.end(1);
    return VSAOGM_OK;
}

int decode_raw(vsaogm_map *m, float *heat, cudaStream_t st)
{
    int rc = memory_norms(m, st);
    if (rc) return rc;
    if (m->cfg.decode_prec != VSAOGM_DECODE_FP32) return decode_tensor_cores(m, heat, st);
    StageScope sc(m, VSAOGM_STAGE_DECODE, st);
    // ordered encoding 0 is below every float: the running maximum starts empty
    cudaError_t e = cudaMemsetAsync(m->maxima, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_error(e, "decode");
    decode_fp32_kernel<<<m->n_dblocks, 256, 0, st>>>(m->dblocks, m->omega, m->inv_norm, m->nu,
                                                    m->cfg.D, m->cfg.grid_w, m->cfg.grid_h,
                                                    m->col_off, m->row_off, heat, m->maxima);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "decode: fp32");
    sc.end(1);
    return VSAOGM_OK;
}

int apply_nonlinearity(vsaogm_map *m, float *heat, cudaStream_t st)
{
    StageScope sc(m, VSAOGM_STAGE_NONLINEAR, st);
    size_t cells = (size_t)m->cfg.grid_w * m->cfg.grid_h;
    int blocks = (int)std::min<size_t>((2 * cells + 255) / 256, 152 * 16);
    nonlinear_kernel<<<blocks, 256, 0, st>>>(heat, cells, m->maxima);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "decode: non-linearity");
    sc.end(1);
    return VSAOGM_OK;
}

int add_memories(float2 *dst, const float2 *src, int64_t count, cudaStream_t st)
{
    int blocks = (int)std::min<int64_t>((count + 255) / 256, 152 * 16);
    add_kernel<<<blocks, 256, 0, st>>>(dst, src, (size_t)count);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VSAOGM_OK : cuda_error(e, "fuse");
}

}  // namespace vsaogm_impl
