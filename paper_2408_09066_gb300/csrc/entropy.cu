// Entropy information extraction (Algorithm 2, Eq. entropy-mask and the
// localized Shannon entropy), softmax over the two classes (Eq. softmax), the
// probabilistic signed difference (Eq. psd) and the threshold (Eq.
// classification), fused in one stencil kernel.
//
// A CTA owns a 32 x 32 block of output cells.  It stages the summand
// h = -P_hat ln P_hat (0 for P_hat = 0) of both classes over the block plus a
// halo of R = max(r_occ, r_emp) cells in shared memory (zero outside the grid,
// which is the same as skipping off-grid neighbours), then sums each cell's
// disk row by row using the exact integer half-widths of the disk.  With raw
// input the non-linearity (P / max P)^2 of Eq. non-linearities is applied while
// staging, so P_hat never makes a round trip through HBM.
#include <algorithm>

#include "internal.cuh"

namespace vsaogm_impl {
namespace {

constexpr int kTB = 32;                       // output cells per block edge
constexpr int kSW = kTB + 2 * kMaxRadius;     // staged edge (64)
constexpr int kSP = kSW + 1;                  // padded row stride

struct DiskParams {
    int r[2];                          // radius per class (0 = empty, 1 = occupied)
    int hw[2][2 * kMaxRadius + 1];     // half-width per dy, -1 outside the disk
};

__global__ void __launch_bounds__(256) entropy_kernel(const float *__restrict__ heat, int W, int H,
                                                      int raw, const unsigned *__restrict__ maxima,
                                                      DiskParams dp, float rho,
                                                      float *__restrict__ occ,
                                                      float *__restrict__ ogm,
                                                      uint8_t *__restrict__ cls)
{
    __shared__ float sh[2][kSW][kSP];
    const int R = max(dp.r[0], dp.r[1]);
    const int x0 = blockIdx.x * kTB, y0 = blockIdx.y * kTB;
    const int edge = kTB + 2 * R;
    float inv[2] = {1.f, 1.f};
    if (raw) {
        for (int c = 0; c < 2; ++c) {
            float m = ordered_to_float(maxima[c]);
            inv[c] = m > 0.f ? 1.0f / m : 0.f;
        }
    }
    const size_t cells = (size_t)W * H;
    for (int c = 0; c < 2; ++c) {
        for (int e = threadIdx.x; e < edge * edge; e += blockDim.x) {
            int ly = e / edge, lx = e % edge;
            int y = y0 - R + ly, x = x0 - R + lx;
            float h = 0.f;
            if (x >= 0 && x < W && y >= 0 && y < H) {
                float v = heat[c * cells + (size_t)y * W + x];
                if (raw) {
                    v *= inv[c];
                    v = v * v;
                }
                if (v != 0.f) h = -v * logf(v);
            }
            sh[c][ly][lx] = h;
        }
    }
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int q = 0; q < kTB / 8; ++q) {
        int ly = ty + 8 * q;
        int x = x0 + tx, y = y0 + ly;
        if (x >= W || y >= H) continue;
        float Hc[2];
        for (int c = 0; c < 2; ++c) {
            const int r = dp.r[c];
            float s = 0.f;
            for (int dy = -r; dy <= r; ++dy) {
                const int w = dp.hw[c][dy + kMaxRadius];
                const float *row = &sh[c][R + ly + dy][R + tx];
                for (int dx = -w; dx <= w; ++dx) s += row[dx];
            }
            Hc[c] = s;
        }
        // Eq. softmax for two classes, then Eq. psd and Eq. classification
        float pr1 = 1.0f / (1.0f + expf(Hc[0] - Hc[1]));
        float pr0 = 1.0f / (1.0f + expf(Hc[1] - Hc[0]));
        size_t o = (size_t)y * W + x;
        occ[o] = pr1;
        float d = pr1 - pr0;
        if (ogm) ogm[o] = d;
        if (cls) cls[o] = d >= rho ? 1 : 0;
    }
}

}  // namespace

int entropy(vsaogm_map *m, const float *heat, bool raw_input, float *occ, float *ogm,
            uint8_t *cls, cudaStream_t st)
{
    DiskParams dp;
    dp.r[0] = m->cfg.r_emp;
    dp.r[1] = m->cfg.r_occ;
    for (int c = 0; c < 2; ++c)
        for (int d = 0; d < 2 * kMaxRadius + 1; ++d) dp.hw[c][d] = m->r_hw[c][d];
    dim3 grid((m->cfg.grid_w + kTB - 1) / kTB, (m->cfg.grid_h + kTB - 1) / kTB);
    StageScope sc(m, VSAOGM_STAGE_ENTROPY, st);
    entropy_kernel<<<grid, 256, 0, st>>>(heat, m->cfg.grid_w, m->cfg.grid_h, raw_input ? 1 : 0,
                                         m->maxima, dp, m->cfg.rho, occ, ogm, cls);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "entropy");
    sc.end(1);
    return VSAOGM_OK;
}

}  // namespace vsaogm_impl
