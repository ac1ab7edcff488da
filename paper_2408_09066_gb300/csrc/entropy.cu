// Entropy information extraction (Algorithm 2, Eq. entropy-mask and the
// localized Shannon entropy), softmax over the two classes (Eq. softmax), the
// probabilistic signed difference (Eq. psd) and the threshold (Eq.
// classification), fused in one stencil kernel.
//
// A CTA owns a 32 x 32 block of output cells.  It stages the summand
// h = -P_hat ln P_hat (0 for P_hat = 0) of both classes over the block plus a
// halo of R = max(r_occ, r_emp) cells in shared memory (zero outside the grid,
// which is the same as skipping off-grid neighbours), turns every staged row
// into running sums, and sums each cell's disk row by row as differences of
// two running sums at the exact integer half-widths of the disk (2 loads per
// disk row instead of one per disk cell).  With raw input the non-linearity
// (P / max P)^2 of Eq. non-linearities is applied while staging, so P_hat
// never makes a round trip through HBM.  ln, exp and the reciprocals use the
// fast hardware approximations: their errors (about 1e-6 relative) are far
// below the probabilities' 1e-3 tolerance.
#include <algorithm>
#include <utility>

#include "internal.cuh"
#include "sm100.cuh"

namespace vsaogm_impl {
namespace {

constexpr int kTB = 32;                       // output cells per block edge

// Hardware log2 of a normal positive float (the approximate MUFU instruction,
// subnormal inputs flushed; its callers never pass one).
__device__ __forceinline__ float lg2_ftz(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
constexpr int kSW = kTB + 2 * kMaxRadius;     // largest staged edge (64)

struct DiskParams {
    int r[2];                          // radius per class (0 = empty, 1 = occupied)
    int hw[2][2 * kMaxRadius + 1];     // half-width per dy, -1 outside the disk
};

// heat: the class maps of a W x H grid of cells (the whole map, or a decoded
// region of it); the block covers window cells (wx0 + x, wy0 + y) of that
// grid, and writes output (x, y) of the ww x wh window, row stride ww.
// The work of one CTA (the 32 x 32 output cells from window cell (bx0, by0)).
// r: disk radius per class; hw: the disks' half-widths per class and dy, in
// shared memory ([2][2 kMaxRadius + 1], -1 outside the disk).  sh: dynamic
// shared memory of staged_floats(R) floats.
__device__ __forceinline__ void entropy_body(const float *__restrict__ heat, int W, int H, int wx0,
                                             int wy0, int ww, int wh, int raw,
                                             const unsigned *__restrict__ maxima, const int *r_c,
                                             const int *hw, unsigned mode, float rho,
                                             float *__restrict__ occ, float *__restrict__ ogm,
                                             uint8_t *__restrict__ cls, int bx0, int by0,
                                             float *sh)
{
    const unsigned act = mode & VSAOGM_ACT_MASK;
    const bool stencil = act == VSAOGM_ACT_ENTROPY;
    const int R = stencil ? max(r_c[0], r_c[1]) : 0;
    const int x0 = wx0 + bx0, y0 = wy0 + by0;                  // grid coordinates
    // staged row: column 0 holds 0, column 1 + lx the summand at lx (after the
    // prefix pass, the sum of the summands left of and at lx)
    const int edge = kTB + 2 * R, pitch = edge + 1;
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
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // Stage: every load of the thread is issued before any is used (rows
    // warp + 8 i, columns lane + 32 s of the staged square), so their
    // latencies overlap.  Off-grid cells read as 0, whose summand is 0.
    constexpr int kRows = kSW / 8, kStrips = kSW / 32;
    float v[2][kRows][kStrips];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int i = 0; i < kRows; ++i)
#pragma unroll
            for (int q = 0; q < kStrips; ++q) {
                const int ly = warp + 8 * i, lx = lane + 32 * q;
                const int y = y0 - R + ly, x = x0 - R + lx;
                v[c][i][q] = (ly < edge && lx < edge && x >= 0 && x < W && y >= 0 && y < H)
                                 ? __ldg(heat + c * cells + (size_t)y * W + x)
                                 : 0.f;
            }
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int i = 0; i < kRows; ++i) {
            const int ly = warp + 8 * i;
            if (ly >= edge) continue;
            float *row = sh + (c * edge + ly) * pitch;
            if (lane == 0) row[0] = 0.f;
#pragma unroll
            for (int q = 0; q < kStrips; ++q) {
                const int lx = lane + 32 * q;
                if (lx < edge) {
                    float x = v[c][i][q];
                    if (norm) x *= inv[c];
                    if (square) x = x * x;
                    // entropy summand -x ln x (0 for x <= 0); other activations keep x
                    row[1 + lx] = stencil ? (x > 0.f ? -x * __logf(x) : 0.f) : x;
                }
            }
        }
    __syncthreads();
    if (stencil) {
        // running sums along each staged row, one thread per row
        for (int rr = threadIdx.x; rr < 2 * edge; rr += blockDim.x) {
            float *row = sh + rr * pitch + 1;
            float acc = 0.f;
#pragma unroll 8
            for (int lx = 0; lx < edge; ++lx) {
                acc += row[lx];
                row[lx] = acc;
            }
        }
        __syncthreads();
    }
    const int tx = lane, ty = warp;
    for (int q = 0; q < kTB / 8; ++q) {
        int ly = ty + 8 * q;
        int x = bx0 + tx, y = by0 + ly;  // window coordinates of the output cell
        if (x >= ww || y >= wh) continue;
        float Hc[2];
        for (int c = 0; c < 2; ++c) {
            if (!stencil) {
                // per-cell activations of the decoding ablation
                const float u = sh[(c * edge + ly) * pitch + 1 + tx];
                Hc[c] = act == VSAOGM_ACT_RELU      ? fmaxf(u, 0.f)
                        : act == VSAOGM_ACT_TANH    ? tanhf(u)
                        : act == VSAOGM_ACT_SIGMOID ? 1.0f / (1.0f + expf(-u))
                                                    : u;
                continue;
            }
            // the disk as rows dy of half-width w: each row's sum is the
            // difference of two running sums
            const int r = r_c[c];
            const int *hwc = hw + c * (2 * kMaxRadius + 1) + kMaxRadius;
            float acc = 0.f;
            for (int dy = -r; dy <= r; ++dy) {
                const int w = hwc[dy];
                const float *row = sh + (c * edge + R + ly + dy) * pitch + R + tx;
                acc += row[w + 1] - row[-w];
            }
            Hc[c] = acc;
        }
        // Eq. softmax for two classes, then Eq. psd and Eq. classification
        float pr1 = __fdividef(1.0f, 1.0f + __expf(Hc[0] - Hc[1]));
        float pr0 = __fdividef(1.0f, 1.0f + __expf(Hc[1] - Hc[0]));
        size_t o = (size_t)y * ww + x;
        if (!VSAOGM_IN_BOUNDS(o < (size_t)ww * wh)) continue;
        occ[o] = pr1;
        float d = pr1 - pr0;
        if (ogm) ogm[o] = d;
        if (cls) cls[o] = d >= rho ? 1 : 0;
    }
}

// Floats of staged summands for halo R: two classes of (32 + 2R) rows of
// pitch 32 + 2R + 1.
__host__ __device__ inline size_t staged_floats(int R)
{
    return 2 * (size_t)(kTB + 2 * R) * (kTB + 2 * R + 1);
}

constexpr int kHW = 2 * kMaxRadius + 1;

// Half-width of the disk of radius r at row offset dy (Eq. entropy-mask: the
// cells with dx^2 + dy^2 <= r^2), -1 outside the disk.
__host__ __device__ constexpr int disk_hw(int r, int dy)
{
    int w = -1;
    if (dy >= -r && dy <= r)
        while ((w + 1) * (w + 1) + dy * dy <= r * r) ++w;
    return w;
}

// Disk sums of kRowsPerThread vertically adjacent output cells of one column,
// rows ly0 .. ly0 + kRowsPerThread - 1, for both classes at once (the staged
// sums are float pairs: class 0, class 1).  Staged row ly0 + T (T in [-R, R +
// kRowsPerThread - 1]) enters output row Q at offset dy = T - Q with the
// disk's half-width w at dy, as the difference of two running sums; `base`
// points at the column of output row ly0.  Offsets and half-widths are
// template constants, so a (row, half-width) difference that several of the
// outputs share is loaded and formed once.
constexpr int kRowsPerThread = 8;
template <int R, int PITCH, int T, int Q>
__device__ __forceinline__ void disk_term(const float2 *base, sm100::f32x2 (&h)[kRowsPerThread])
{
    using namespace sm100;
    constexpr int dy = T - Q;
    if constexpr (dy >= -R && dy <= R) {
        constexpr int w = disk_hw(R, dy);
        static_assert(w >= 0, "rows of the disk only");
        const float2 hi = base[T * PITCH + w + 1], lo = base[T * PITCH - w];
        h[Q] = add2(h[Q], sub2(pack2(hi.x, hi.y), pack2(lo.x, lo.y)));
    }
}
template <int R, int PITCH, int T, int... Q>
__device__ __forceinline__ void disk_row(const float2 *base, sm100::f32x2 (&h)[kRowsPerThread],
                                         std::integer_sequence<int, Q...>)
{
    (disk_term<R, PITCH, T, Q>(base, h), ...);
}
template <int R, int PITCH, int... I>
__device__ __forceinline__ void disk_sums(const float2 *base, sm100::f32x2 (&h)[kRowsPerThread],
                                          std::integer_sequence<int, I...>)
{
    (disk_row<R, PITCH, I - R>(base, h, std::make_integer_sequence<int, kRowsPerThread>{}), ...);
}

// threads per entropy CTA: 4 warps, each thread kRowsPerThread output rows of
// one column of the 32 x 32 block
constexpr int kEntThreads = 32 * (kTB / kRowsPerThread);

// The entropy stencil for the common case of one disk radius R (<= 8) for
// both classes: the same computation as entropy_body with every loop bound,
// staged extent and disk half-width known at compile time, and both classes
// carried together as float pairs in shared memory and in packed f32x2
// arithmetic (one instruction does each step for both).  Staging walks the
// (32 + 2R)^2 staged cells as one flat range (no lane idles on a row's ragged
// end), and each thread sums the disks of kRowsPerThread vertically adjacent
// cells of one column, so the disk rows they share are read once.
template <int R>
__device__ __forceinline__ void entropy_fixed_body(const float *__restrict__ heat, int W, int H,
                                                   int wx0, int wy0, int ww, int wh, int raw,
                                                   const unsigned *__restrict__ maxima,
                                                   unsigned mode, float rho,
                                                   float *__restrict__ occ,
                                                   float *__restrict__ ogm,
                                                   uint8_t *__restrict__ cls, int bx0, int by0,
                                                   float *shf)
{
    using namespace sm100;
    constexpr int E = kTB + 2 * R, PITCH = E + 1, EE = E * E;
    constexpr int SLOTS = (EE + kEntThreads - 1) / kEntThreads;
    static_assert(kTB == 32 && kEntThreads * kRowsPerThread == 32 * kTB,
                  "each warp's lanes cover the block's 32 columns for kRowsPerThread rows");
    float2 *sh = reinterpret_cast<float2 *>(shf);  // [E][PITCH] pairs (class 0, class 1)
    const int x0 = wx0 + bx0, y0 = wy0 + by0;
    float inv[2] = {1.f, 1.f};
    const bool norm = raw && !(mode & VSAOGM_MODE_NO_NORM);
    const bool square = raw && !(mode & VSAOGM_MODE_NO_SQUARE);
    if (norm) {
        for (int c = 0; c < 2; ++c) {
            float m = ordered_to_float(maxima[c]);
            inv[c] = m > 0.f ? 1.0f / m : 0.f;
        }
    }
    const f32x2 INV = pack2(inv[0], inv[1]);
    const f32x2 kNegLn2 = pack2(-0.69314718055994531f, -0.69314718055994531f);
    const size_t cells = (size_t)W * H;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // Stage: staged cell e = ly * E + lx; every load of the thread is issued
    // before any is used.  Off-grid cells read as 0, whose summand is 0; when
    // the whole staged square lies inside the grid (most blocks of a large
    // map) no cell needs that test.
    float v0[SLOTS], v1[SLOTS];
    int so[SLOTS];  // the cell's pair in shared memory
    const bool inside = x0 - R >= 0 && y0 - R >= 0 && x0 - R + E <= W && y0 - R + E <= H;
    if (inside) {
        const float *g0 = heat + ((size_t)(y0 - R) * W + (x0 - R));
        const float *g1 = g0 + cells;
#pragma unroll
        for (int i = 0; i < SLOTS; ++i) {
            const int e = tid + kEntThreads * i;
            const int ly = e / E, lx = e - ly * E;
            const bool ok = (i + 1) * kEntThreads <= EE || e < EE;
            const int off = ly * W + lx;
            v0[i] = ok ? __ldg(g0 + off) : 0.f;
            v1[i] = ok ? __ldg(g1 + off) : 0.f;
            so[i] = ok ? ly * PITCH + 1 + lx : -1;
        }
    } else {
#pragma unroll
        for (int i = 0; i < SLOTS; ++i) {
            const int e = tid + kEntThreads * i;
            const int ly = e / E, lx = e - ly * E;
            const int y = y0 - R + ly, x = x0 - R + lx;
            const bool ok = e < EE && x >= 0 && x < W && y >= 0 && y < H;
            const size_t g = (size_t)y * W + x;
            v0[i] = ok ? __ldg(heat + g) : 0.f;
            v1[i] = ok ? __ldg(heat + cells + g) : 0.f;
            so[i] = e < EE ? ly * PITCH + 1 + lx : -1;
        }
    }
#pragma unroll
    for (int i = 0; i < SLOTS; ++i) {
        if (so[i] >= 0) {
            f32x2 a = pack2(v0[i], v1[i]);
            if (norm) a = mul2(a, INV);
            if (square) a = mul2(a, a);
            // -a ln a = a log2(a) (-ln 2), 0 for a <= 0 (Eq. entropy summand)
            const float2 af = unpack2(a);
            if (square) {
                // a >= 0: log2 of max(a, 2^-100) is finite, and for a = 0 the
                // product is 0 (below 2^-100 the summand is under 1e-28 anyway)
                const float2 h = unpack2(mul2(mul2(a, pack2(lg2_ftz(fmaxf(af.x, 7.9e-31f)),
                                                            lg2_ftz(fmaxf(af.y, 7.9e-31f)))),
                                              kNegLn2));
                sh[so[i]] = h;
            } else {
                const float2 h =
                    unpack2(mul2(mul2(a, pack2(__log2f(af.x), __log2f(af.y))), kNegLn2));
                sh[so[i]] = make_float2(af.x > 0.f ? h.x : 0.f, af.y > 0.f ? h.y : 0.f);
            }
        }
    }
    if (tid < E) sh[tid * PITCH] = make_float2(0.f, 0.f);
    __syncthreads();
    // running sums along each staged row, one thread per row
    if (tid < E) {
        float2 *row = sh + tid * PITCH + 1;
        f32x2 acc = pack2(0.f, 0.f);
#pragma unroll
        for (int lx = 0; lx < E; ++lx) {
            const float2 t = row[lx];
            acc = add2(acc, pack2(t.x, t.y));
            row[lx] = unpack2(acc);
        }
    }
    __syncthreads();
    const int ly0 = kRowsPerThread * warp;
    f32x2 Hc[kRowsPerThread];
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) Hc[q] = pack2(0.f, 0.f);
    disk_sums<R, PITCH>(sh + (R + ly0) * PITCH + R + lane, Hc,
                        std::make_integer_sequence<int, 2 * R + kRowsPerThread>{});
    const int x = bx0 + lane;
    // Eq. softmax for two classes: Pr(psi = 1) = 1 / (1 + e^(H0 - H1)) and
    // Pr(psi = 0) = 1 - Pr(psi = 1), so the signed difference of Eq. psd is
    // 2 Pr(psi = 1) - 1; then Eq. classification
    float *occ_row = occ + ((size_t)(by0 + ly0) * ww + x);
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
        const int y = by0 + ly0 + q;
        if (x >= ww || y >= wh) continue;
        const float2 hq = unpack2(Hc[q]);
        const float pr1 = __fdividef(1.0f, 1.0f + __expf(hq.x - hq.y));
        const float d = fmaf(2.0f, pr1, -1.0f);
        const int o = q * ww;  // from the thread's first output cell
        if (!VSAOGM_IN_BOUNDS((size_t)y * ww + x < (size_t)ww * wh)) continue;
        occ_row[o] = pr1;
        if (ogm) ogm[(occ_row - occ) + o] = d;
        if (cls) cls[(occ_row - occ) + o] = d >= rho ? 1 : 0;
    }
}

// Radius of the fixed-radius stencil, or -1 when the generic one is needed
// (another activation, two radii, or a radius above 8).
__host__ inline int fixed_radius(unsigned mode, int r0, int r1)
{
    if ((mode & VSAOGM_ACT_MASK) != VSAOGM_ACT_ENTROPY || r0 != r1 || r0 > 8) return -1;
    return r0;
}

template <int R>
__global__ void __launch_bounds__(kEntThreads) entropy_fixed_kernel(const float *__restrict__ heat, int W,
                                                            int H, int wx0, int wy0, int ww, int wh,
                                                            int raw,
                                                            const unsigned *__restrict__ maxima,
                                                            unsigned mode, float rho,
                                                            float *__restrict__ occ,
                                                            float *__restrict__ ogm,
                                                            uint8_t *__restrict__ cls)
{
    extern __shared__ float sh_dyn[];
    entropy_fixed_body<R>(heat, W, H, wx0, wy0, ww, wh, raw, maxima, mode, rho, occ, ogm, cls,
                          blockIdx.x * kTB, blockIdx.y * kTB, sh_dyn);
}

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
    extern __shared__ float sh_dyn[];
    __shared__ int hw[2 * kHW];
    if (threadIdx.x < 2 * kHW) hw[threadIdx.x] = dp.hw[threadIdx.x / kHW][threadIdx.x % kHW];
    __syncthreads();
    entropy_body(heat, W, H, wx0, wy0, ww, wh, raw, maxima, dp.r, hw, mode, rho, occ, ogm, cls,
                 blockIdx.x * kTB, blockIdx.y * kTB, sh_dyn);
}

// Every map of a batch in one launch: CTA q takes block q of the list of all
// maps' 32 x 32 blocks (map by binary search over the first block of each).
__global__ void __launch_bounds__(256) entropy_batch_kernel(const __grid_constant__ BatchOutTable tab)
{
    extern __shared__ float sh_dyn[];
    const int q = blockIdx.x;
    int lo = 0, hi = tab.n_maps - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tab.m[mid].blk_begin <= q) lo = mid; else hi = mid - 1;
    }
    const BatchMapOut &M = tab.m[lo];
    const int local = q - M.blk_begin, bxn = (M.W + kTB - 1) / kTB;
    const int bx0 = (local % bxn) * kTB, by0 = (local / bxn) * kTB;
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
                 M.ogm, nullptr, bx0, by0, sh_dyn);
}

template <int R>
__global__ void __launch_bounds__(kEntThreads) entropy_fixed_batch_kernel(const __grid_constant__ BatchOutTable tab)
{
    extern __shared__ float sh_dyn[];
    const int q = blockIdx.x;
    int lo = 0, hi = tab.n_maps - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tab.m[mid].blk_begin <= q) lo = mid; else hi = mid - 1;
    }
    const BatchMapOut &M = tab.m[lo];
    const int local = q - M.blk_begin, bxn = (M.W + kTB - 1) / kTB;
    entropy_fixed_body<R>(M.heat, M.W, M.H, 0, 0, M.W, M.H, 1, M.maxima, M.mode, M.rho, M.occ,
                          M.ogm, nullptr, (local % bxn) * kTB, (local / bxn) * kTB, sh_dyn);
}

}  // namespace

int launch_entropy_batch(const BatchOutTable &tab, cudaStream_t st)
{
    int blocks = 0, R = 0;
    for (int i = 0; i < tab.n_maps; ++i) {
        const BatchMapOut &M = tab.m[i];
        if (M.blk_begin != blocks) return set_error(VSAOGM_E_INVAL, "batch entropy: block table");
        blocks += ((M.W + kTB - 1) / kTB) * ((M.H + kTB - 1) / kTB);
        if ((M.mode & VSAOGM_ACT_MASK) == VSAOGM_ACT_ENTROPY) R = std::max(R, std::max(M.r[0], M.r[1]));
    }
    // one radius for both classes of every map: the fixed-radius stencil
    int fixed = tab.n_maps > 0 ? fixed_radius(tab.m[0].mode, tab.m[0].r[0], tab.m[0].r[1]) : -1;
    for (int i = 1; i < tab.n_maps && fixed >= 0; ++i)
        if (fixed_radius(tab.m[i].mode, tab.m[i].r[0], tab.m[i].r[1]) != fixed) fixed = -1;
    const size_t smem = staged_floats(R) * sizeof(float);
    switch (fixed) {
#define VSAOGM_FIXED_BATCH(RR) \
    case RR: entropy_fixed_batch_kernel<RR><<<blocks, kEntThreads, smem, st>>>(tab); break;
        VSAOGM_FIXED_BATCH(0) VSAOGM_FIXED_BATCH(1) VSAOGM_FIXED_BATCH(2) VSAOGM_FIXED_BATCH(3)
        VSAOGM_FIXED_BATCH(4) VSAOGM_FIXED_BATCH(5) VSAOGM_FIXED_BATCH(6) VSAOGM_FIXED_BATCH(7)
        VSAOGM_FIXED_BATCH(8)
#undef VSAOGM_FIXED_BATCH
        default: entropy_batch_kernel<<<blocks, 256, smem, st>>>(tab);
    }
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
    const unsigned act = m->cfg.decode_mode & VSAOGM_ACT_MASK;
    const int R = act == VSAOGM_ACT_ENTROPY ? std::max(dp.r[0], dp.r[1]) : 0;
    const size_t smem = staged_floats(R) * sizeof(float);
    const int fixed = fixed_radius(m->cfg.decode_mode, dp.r[0], dp.r[1]);
    switch (fixed) {
#define VSAOGM_FIXED(RR)                                                                          \
    case RR:                                                                                      \
        entropy_fixed_kernel<RR><<<grid, kEntThreads, smem, st>>>(heat, r.w(), r.h(), win.x0 - r.x0,      \
                                                          win.y0 - r.y0, win.w(), win.h(),        \
                                                          raw_input ? 1 : 0, m->maxima,           \
                                                          m->cfg.decode_mode, m->cfg.rho, occ,    \
                                                          ogm, cls);                              \
        break;
        VSAOGM_FIXED(0) VSAOGM_FIXED(1) VSAOGM_FIXED(2) VSAOGM_FIXED(3) VSAOGM_FIXED(4)
        VSAOGM_FIXED(5) VSAOGM_FIXED(6) VSAOGM_FIXED(7) VSAOGM_FIXED(8)
#undef VSAOGM_FIXED
        default:
            entropy_kernel<<<grid, 256, smem, st>>>(heat, r.w(), r.h(), win.x0 - r.x0,
                                                    win.y0 - r.y0, win.w(), win.h(),
                                                    raw_input ? 1 : 0, m->maxima, dp,
                                                    m->cfg.decode_mode, m->cfg.rho, occ, ogm, cls);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "entropy");
    sc.end(1);
    return VSAOGM_OK;
}

VSAOGM_CHECK_TU(entropy)

}  // namespace vsaogm_impl
