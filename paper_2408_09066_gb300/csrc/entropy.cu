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

// heat: the class maps of a W x H grid of cells (the whole map, or a decoded
// region of it); the block covers window cells (wx0 + x, wy0 + y) of that
// grid, and writes output (x, y) of the ww x wh window, row stride ww.
__global__ void __launch_bounds__(256) entropy_kernel(const float *__restrict__ heat, int W, int H,
                                                      int wx0, int wy0, int ww, int wh, int raw,
                                                      const unsigned *__restrict__ maxima,
                                                      DiskParams dp, unsigned mode, float rho,
                                                      float *__restrict__ occ,
                                                      float *__restrict__ ogm,
                                                      uint8_t *__restrict__ cls)
{
    __shared__ float sh[2][kSW][kSP];
    const unsigned act = mode & VSAOGM_ACT_MASK;
    const bool stencil = act == VSAOGM_ACT_ENTROPY;
    const int R = stencil ? max(dp.r[0], dp.r[1]) : 0;
    const int bx0 = blockIdx.x * kTB, by0 = blockIdx.y * kTB;  // window coordinates
    const int x0 = wx0 + bx0, y0 = wy0 + by0;                  // grid coordinates
    const int edge = kTB + 2 * R;
    float inv[2] = {1.f, 1.f};
    const bool norm = raw && !(mode & VSAOGM_MODE_NO_NORM);
    const bool square = raw && !(mode & VSAOGM_MODE_NO_SQUARE);
    if (norm) {
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
                if (norm) v *= inv[c];
                if (square) v = v * v;
                // entropy summand -v ln v (0 for v <= 0); other activations keep v
                h = stencil ? (v > 0.f ? -v * logf(v) : 0.f) : v;
            }
            sh[c][ly][lx] = h;
        }
    }
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int q = 0; q < kTB / 8; ++q) {
        int ly = ty + 8 * q;
        int x = bx0 + tx, y = by0 + ly;  // window coordinates of the output cell
        if (x >= ww || y >= wh) continue;
        float Hc[2];
        for (int c = 0; c < 2; ++c) {
            if (!stencil) {
                // per-cell activations of the decoding ablation
                const float v = sh[c][ly][tx];
                Hc[c] = act == VSAOGM_ACT_RELU      ? fmaxf(v, 0.f)
                        : act == VSAOGM_ACT_TANH    ? tanhf(v)
                        : act == VSAOGM_ACT_SIGMOID ? 1.0f / (1.0f + expf(-v))
                                                    : v;
                continue;
            }
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
        size_t o = (size_t)y * ww + x;
        occ[o] = pr1;
        float d = pr1 - pr0;
        if (ogm) ogm[o] = d;
        if (cls) cls[o] = d >= rho ? 1 : 0;
    }
}

}  // namespace

int entropy(vsaogm_map *m, const float *heat, Region r, Region win, bool raw_input, float *occ,
            float *ogm, uint8_t *cls, cudaStream_t st)
{
    DiskParams dp;
    dp.r[0] = m->cfg.r_emp;
    dp.r[1] = m->cfg.r_occ;
    for (int c = 0; c < 2; ++c)
        for (int d = 0; d < 2 * kMaxRadius + 1; ++d) dp.hw[c][d] = m->r_hw[c][d];
    dim3 grid((win.w() + kTB - 1) / kTB, (win.h() + kTB - 1) / kTB);
    StageScope sc(m, VSAOGM_STAGE_ENTROPY, st);
    entropy_kernel<<<grid, 256, 0, st>>>(heat, r.w(), r.h(), win.x0 - r.x0, win.y0 - r.y0,
                                         win.w(), win.h(), raw_input ? 1 : 0, m->maxima, dp,
                                         m->cfg.decode_mode, m->cfg.rho, occ, ogm, cls);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "entropy");
    sc.end(1);
    return VSAOGM_OK;
}

}  // namespace vsaogm_impl
