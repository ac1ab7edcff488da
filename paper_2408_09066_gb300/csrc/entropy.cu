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
// The work of one CTA (the 32 x 32 output cells from window cell (bx0, by0)).
// r: disk radius per class; hw: the disks' half-widths per class and dy, in
// shared memory ([2][2 kMaxRadius + 1], -1 outside the disk).
__device__ __forceinline__ void entropy_body(const float *__restrict__ heat, int W, int H, int wx0,
                                             int wy0, int ww, int wh, int raw,
                                             const unsigned *__restrict__ maxima, const int *r_c,
                                             const int *hw, unsigned mode, float rho,
                                             float *__restrict__ occ, float *__restrict__ ogm,
                                             uint8_t *__restrict__ cls, int bx0, int by0)
{
    __shared__ float sh[2][kSW][kSP];
    const unsigned act = mode & VSAOGM_ACT_MASK;
    const bool stencil = act == VSAOGM_ACT_ENTROPY;
    const int R = stencil ? max(r_c[0], r_c[1]) : 0;
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
            const int r = r_c[c];
            float s = 0.f;
            for (int dy = -r; dy <= r; ++dy) {
                const int w = hw[c * (2 * kMaxRadius + 1) + dy + kMaxRadius];
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

constexpr int kHW = 2 * kMaxRadius + 1;

// heat: the class maps of a W x H grid of cells (the whole map, or a decoded
// region of it); the grid of CTAs covers window cells (wx0 + x, wy0 + y) of
// that grid and writes output (x, y) of the ww x wh window, row stride ww.
__global__ void __launch_bounds__(256) entropy_kernel(const float *__restrict__ heat, int W, int H,
                                                      int wx0, int wy0, int ww, int wh, int raw,
                                                      const unsigned *__restrict__ maxima,
                                                      DiskParams dp, unsigned mode, float rho,
                                                      float *__restrict__ occ,
                                                      float *__restrict__ ogm,
                                                      uint8_t *__restrict__ cls)
{
    __shared__ int hw[2 * kHW];
    if (threadIdx.x < 2 * kHW) hw[threadIdx.x] = dp.hw[threadIdx.x / kHW][threadIdx.x % kHW];
    __syncthreads();
    entropy_body(heat, W, H, wx0, wy0, ww, wh, raw, maxima, dp.r, hw, mode, rho, occ, ogm, cls,
                 blockIdx.x * kTB, blockIdx.y * kTB);
}

// Every map of a batch in one launch: blockIdx.z is the map; the grid covers
// the largest map and CTAs beyond a map's extent return at once.
__global__ void __launch_bounds__(256) entropy_batch_kernel(const __grid_constant__ BatchOutTable tab)
{
    const BatchMapOut &M = tab.m[blockIdx.z];
    const int bx0 = blockIdx.x * kTB, by0 = blockIdx.y * kTB;
    if (bx0 >= M.W || by0 >= M.H) return;
    __shared__ int hw[2 * kHW];
    if (threadIdx.x < 2 * kHW) {
        // half-width of the disk of class c at row offset dy (Eq. entropy-mask)
        const int c = threadIdx.x / kHW, dy = threadIdx.x % kHW - kMaxRadius, r = M.r[c];
        int w = -1;
        if (dy >= -r && dy <= r)
            while ((w + 1) * (w + 1) + dy * dy <= r * r) ++w;
        hw[threadIdx.x] = w;
    }
    __syncthreads();
    entropy_body(M.heat, M.W, M.H, 0, 0, M.W, M.H, 1, M.maxima, M.r, hw, M.mode, M.rho, M.occ,
                 M.ogm, nullptr, bx0, by0);
}

}  // namespace

int launch_entropy_batch(const BatchOutTable &tab, int w_max, int h_max, cudaStream_t st)
{
    dim3 grid((w_max + kTB - 1) / kTB, (h_max + kTB - 1) / kTB, tab.n_maps);
    entropy_batch_kernel<<<grid, 256, 0, st>>>(tab);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VSAOGM_OK : cuda_error(e, "batch entropy");
}

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
