// Host runtime and C ABI of libvsaogm.so: map lifetime, configuration,
// axis-frequency draw, tile and cell geometry, and the entry points declared
// in include/vsaogm.h.  Kernels live in encode.cu, decode.cu and entropy.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

using namespace vsaogm_impl;

namespace {
thread_local char g_err[512] = "";
std::mutex g_alloc_mu;
std::unordered_map<void *, size_t> g_alloc_live;  // device blocks the library holds
long long g_alloc_bytes = 0;
thread_local int g_alloc_count = 0;  // allocations since the entry point began
}

namespace vsaogm_impl {

void alloc_scope_begin() { g_alloc_count = 0; }

cudaError_t dev_malloc(void **p, size_t bytes)
{
    *p = nullptr;
    ++g_alloc_count;
    if (const char *v = getenv("VSAOGM_FAIL_ALLOC"))
        if (atoi(v) == g_alloc_count) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    g_alloc_live[*p] = bytes;
    g_alloc_bytes += (long long)bytes;
    return e;
}

cudaError_t dev_free(void *p)
{
    if (!p) return cudaSuccess;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mu);
        auto it = g_alloc_live.find(p);
        if (it != g_alloc_live.end()) {
            g_alloc_bytes -= (long long)it->second;
            g_alloc_live.erase(it);
        }
    }
    return cudaFree(p);
}

long long device_bytes_held()
{
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    return g_alloc_bytes;
}

int set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_error(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_error(VSAOGM_E_NOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return set_error(VSAOGM_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Grows b to at least `bytes` (never shrinks).  Growing frees the old block,
// which synchronises the device.
int ensure(DevBuf &b, size_t bytes)
{
    if (b.bytes >= bytes) return VSAOGM_OK;
    if (b.ptr) dev_free(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
    size_t want = bytes + bytes / 8 + 256;  // headroom against repeated growth
    cudaError_t e = dev_malloc(&b.ptr, want);
    if (e != cudaSuccess) {
        b.ptr = nullptr;
        return cuda_error(e, "scratch allocation");
    }
    b.bytes = want;
    return VSAOGM_OK;
}

static cudaEvent_t take_event(vsaogm_map *m)
{
    auto &pool = m->timer.free_events;
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

StageScope::StageScope(vsaogm_map *m, int stage, cudaStream_t st) : m_(m), stage_(stage), st_(st)
{
    if (m->timer.enabled) {
        a_ = take_event(m);
        if (a_ && cudaEventRecord(a_, st) != cudaSuccess) {
            m->timer.free_events.push_back(a_);
            a_ = nullptr;
        }
    }
}

void StageScope::end(int kernels)
{
    m_->timer.launches[stage_] += kernels;
    if (a_) {
        cudaEvent_t b = take_event(m_);
        if (b && cudaEventRecord(b, st_) == cudaSuccess) {
            m_->timer.pending.push_back({stage_, a_, b});
        } else {
            if (b) m_->timer.free_events.push_back(b);
            m_->timer.free_events.push_back(a_);
        }
        a_ = nullptr;
    }
    done_ = true;
}

StageScope::~StageScope()
{
    if (a_) m_->timer.free_events.push_back(a_);
}

void free_scratch(Scratch &ws)
{
    DevBuf *bufs[] = {&ws.blk_hist, &ws.seg_meta,  &ws.chunks,    &ws.sorted,
                      &ws.partial,  &ws.stage_xy,  &ws.stage_lab, &ws.stage_heat,
                      &ws.stage_occ, &ws.dec_partial, &ws.map_heat};
    for (DevBuf *b : bufs) {
        if (b->ptr) dev_free(b->ptr);
        b->ptr = nullptr;
        b->bytes = 0;
    }
}

}  // namespace vsaogm_impl

namespace {

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) as a counter-based
// generator: output i of the stream seeded with s is mix(s + (i + 1) * gamma),
// gamma = 0x9E3779B97F4A7C15, with the variant-13 mixing function.
uint64_t splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Largest float not above the double v (so that, for a float x, x > v holds
// exactly when x > round_down(v)).
float round_down_f32(double v)
{
    float f = (float)v;
    if ((double)f > v) f = std::nextafter(f, -INFINITY);
    return f;
}


void free_map(vsaogm_map *m)
{
    if (!m) return;
    void *ptrs[] = {m->nu, m->omega, m->inv_norm, m->maxima, m->rejected, m->enc_cnt, m->bnd_x_lo,
                    m->bnd_y_lo, m->centre_x, m->centre_y, m->col_tile, m->row_tile,
                    m->col_off, m->row_off, m->status, m->patch_cx[0], m->patch_cy[0],
                    m->patch_cx[1], m->patch_cy[1], m->tc_rot, m->tc_xtab, m->tc_xtmap};
    for (void *p : ptrs)
        if (p) dev_free(p);
    free_scratch(m->ws);
    for (cudaEvent_t e : m->timer.free_events) cudaEventDestroy(e);
    for (auto &p : m->timer.pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    free(m->host_nu);
    delete m;
}

int validate(const vsaogm_config *c)
{
    if (!c) return set_error(VSAOGM_E_INVAL, "config is NULL");
    if (c->D < 1 || c->D > (1 << 22)) return set_error(VSAOGM_E_INVAL, "D must be in [1, 2^22]");
    if (c->grid_w < 1 || c->grid_h < 1 || c->grid_w > (1 << 16) || c->grid_h > (1 << 16))
        return set_error(VSAOGM_E_INVAL, "grid_w, grid_h must be in [1, 65536]");
    if (!(c->resolution > 0.0f) || !std::isfinite(c->resolution))
        return set_error(VSAOGM_E_INVAL, "resolution must be positive and finite");
    if (!std::isfinite(c->x_min) || !std::isfinite(c->y_min))
        return set_error(VSAOGM_E_INVAL, "x_min, y_min must be finite");
    if (c->tiles_x < 1 || c->tiles_y < 1 || c->tiles_x > c->grid_w || c->tiles_y > c->grid_h)
        return set_error(VSAOGM_E_INVAL, "tiles per axis must be in [1, cells on that axis]");
    if ((int64_t)c->tiles_x * c->tiles_y > kMaxTiles)
        return set_error(VSAOGM_E_INVAL, "tiles_x * tiles_y must be <= %d", kMaxTiles);
    if (!(c->length_scale > 0.0f) || !std::isfinite(c->length_scale))
        return set_error(VSAOGM_E_INVAL, "length_scale must be positive and finite");
    if (c->r_occ < 0 || c->r_emp < 0 || c->r_occ > kMaxRadius || c->r_emp > kMaxRadius)
        return set_error(VSAOGM_E_INVAL, "disk radii must be in [0, %d]", kMaxRadius);
    if (!std::isfinite(c->rho)) return set_error(VSAOGM_E_INVAL, "rho must be finite");
    if (c->decode_prec != VSAOGM_DECODE_FP32 && c->decode_prec != VSAOGM_DECODE_BF16X3 &&
        c->decode_prec != VSAOGM_DECODE_FP16X3 && c->decode_prec != VSAOGM_DECODE_FP8X3)
        return set_error(VSAOGM_E_INVAL, "unknown decode_prec %d", c->decode_prec);
    if (c->flags & ~(VSAOGM_FLAG_CHECKED | VSAOGM_FLAG_ATOMIC | VSAOGM_FLAG_WINDOW_MAP_MAX))
        return set_error(VSAOGM_E_INVAL, "unknown flags 0x%x", c->flags);
    if ((c->decode_mode & ~(VSAOGM_MODE_NO_NORM | VSAOGM_MODE_NO_SQUARE | VSAOGM_ACT_MASK)) ||
        (c->decode_mode & VSAOGM_ACT_MASK) > VSAOGM_ACT_NONE)
        return set_error(VSAOGM_E_INVAL, "unknown decode_mode 0x%x", c->decode_mode);
    return VSAOGM_OK;
}

// One axis of the tiling (Sec. III-B3) and its cell table.
struct AxisHost {
    std::vector<float> bnd_lo;     // tiles - 1
    std::vector<double> centre;    // tiles
    std::vector<int> cell_tile;    // cells
    std::vector<float> cell_off;   // cells
    std::vector<int> first, last;  // per tile: first cell and one past the last
};

// FP64 values as float pairs hi + lo, hi = f32(v), lo = f32(v - hi): about 48
// significant bits, for the sort's offsets from tile centres without FP64.
std::vector<float2> centre_pairs(const std::vector<double> &v)
{
    std::vector<float2> out;
    for (double c : v) {
        const float hi = (float)c;
        out.push_back(make_float2(hi, (float)(c - (double)hi)));
    }
    return out;
}

AxisHost build_axis(int cells, int tiles, double res, double lo)
{
    AxisHost a;
    double tw = (double)cells * res / (double)tiles;
    for (int t = 1; t < tiles; ++t) a.bnd_lo.push_back(round_down_f32(lo + (double)t * tw));
    for (int t = 0; t < tiles; ++t) a.centre.push_back(lo + ((double)t + 0.5) * tw);
    a.first.assign(tiles, cells);
    a.last.assign(tiles, 0);
    for (int i = 0; i < cells; ++i) {
        double x = lo + ((double)i + 0.5) * res;
        // Algorithm 1 on a regular lattice: the nearest centre along this axis,
        // the lower tile on an exact tie (x equal to a boundary).
        int t = 0;
        while (t + 1 < tiles && x > lo + (double)(t + 1) * tw) ++t;
        a.cell_tile.push_back(t);
        a.cell_off.push_back((float)(x - a.centre[t]));
        if (i < a.first[t]) a.first[t] = i;
        if (i + 1 > a.last[t]) a.last[t] = i + 1;
    }
    return a;
}

template <typename T>
int upload(T **dst, const std::vector<T> &v)
{
    size_t bytes = sizeof(T) * (v.empty() ? 1 : v.size());
    cudaError_t e = dev_malloc((void **)dst, bytes);
    if (e != cudaSuccess) {
        *dst = nullptr;
        return cuda_error(e, "map allocation");
    }
    if (!v.empty()) {
        e = cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_error(e, "map upload");
    }
    return VSAOGM_OK;
}

// Disk half-widths: for dy in [-r, r], the largest dx with dx^2 + dy^2 <= r^2
// (Eq. entropy-mask with the distance of the following equation, inclusive).
void disk_half_widths(int r, int *hw)
{
    for (int dy = -kMaxRadius; dy <= kMaxRadius; ++dy) {
        int w = -1;
        if (dy >= -r && dy <= r)
            while ((w + 1) * (w + 1) + dy * dy <= r * r) ++w;
        hw[dy + kMaxRadius] = w;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
#define VSA_TRY(expr)                      \
    do {                                   \
        int rc_ = (expr);                  \
        if (rc_ != VSAOGM_OK) return rc_;  \
    } while (0)

#define VSA_CUDA(expr, what)                                   \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) return cuda_error(e_, what);    \
    } while (0)


extern "C" {

const char *vsaogm_last_error(void) { return g_err; }

int vsaogm_device_bytes(int64_t *bytes)
{
    if (!bytes) return set_error(VSAOGM_E_INVAL, "bytes is NULL");
    *bytes = (int64_t)device_bytes_held();
    return VSAOGM_OK;
}

void vsaogm_config_default(vsaogm_config *c)
{
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->D = 8192;
    c->grid_w = c->grid_h = 400;
    c->resolution = 0.1f;
    c->x_min = c->y_min = -20.0f;
    c->tiles_x = c->tiles_y = 4;
    c->length_scale = 0.1f;
    c->r_occ = c->r_emp = 3;
    c->rho = 0.0f;
    c->seed = 0;
    c->decode_prec = VSAOGM_DECODE_FP32;
    c->flags = 0;
}

int vsaogm_create(const vsaogm_config *cfg, vsaogm_map **out)
{
    alloc_scope_begin();
    if (!out) return set_error(VSAOGM_E_INVAL, "out is NULL");
    *out = nullptr;
    VSA_TRY(validate(cfg));
    vsaogm_map *m = new (std::nothrow) vsaogm_map();
    if (!m) return set_error(VSAOGM_E_NOMEM, "host allocation");
    m->cfg = *cfg;
    int rc = VSAOGM_OK;
    do {
        if (cudaGetDevice(&m->device) != cudaSuccess) {
            rc = set_error(VSAOGM_E_CUDA, "no CUDA device");
            break;
        }
        const int D = cfg->D;
        m->T = cfg->tiles_x * cfg->tiles_y;
        m->S = 2 * m->T;
        // Axis frequencies (Sec. III-B2), drawn once on the host.
        m->host_nu = (float *)malloc(sizeof(float) * 2 * (size_t)D);
        if (!m->host_nu) {
            rc = set_error(VSAOGM_E_NOMEM, "host allocation");
            break;
        }
        const double half_band = 0.5 / (double)cfg->length_scale;
        for (int k = 0; k < D; ++k) {
            double ux = (double)(splitmix64(cfg->seed, 2u * (uint64_t)k) >> 11) * 0x1.0p-53;
            double uy = (double)(splitmix64(cfg->seed, 2u * (uint64_t)k + 1u) >> 11) * 0x1.0p-53;
            m->host_nu[k] = (float)((2.0 * ux - 1.0) * half_band);
            m->host_nu[D + k] = (float)((2.0 * uy - 1.0) * half_band);
            m->nu_max[0] = std::max(m->nu_max[0], std::fabs(m->host_nu[k]));
            m->nu_max[1] = std::max(m->nu_max[1], std::fabs(m->host_nu[D + k]));
        }
        // encode kernel family (tuning overrides through the environment)
        m->encode_packed = 1;
        m->encode_poly_pairs = 0;
        m->encode_poly_warps = -1;  // automatic share of polynomial phasors
        if (const char *v = getenv("VSAOGM_ENCODE_PACKED")) m->encode_packed = atoi(v) != 0;
        if (const char *v = getenv("VSAOGM_ENCODE_POLY"))
            m->encode_poly_pairs = std::max(0, std::min(3, atoi(v)));
        if (const char *v = getenv("VSAOGM_ENCODE_POLY_WARPS"))
            m->encode_poly_warps = std::max(-1, std::min(16, atoi(v)));
        // failure test of the bounded waits (see vsaogm_status)
        m->debug_wait_ns = 0;
        m->mem_gen = 0;
        m->map_heat_gen = ~0ull;
        if (const char *v = getenv("VSAOGM_DEBUG_WAIT_NS"))
            m->debug_wait_ns = (uint64_t)std::max(0LL, std::min(1000000000LL, atoll(v)));
        std::vector<float> nu(m->host_nu, m->host_nu + 2 * (size_t)D);
        if ((rc = upload(&m->nu, nu))) break;
        // Tiling and cell tables (Sec. III-B3, Algorithm 1).
        AxisHost ax = build_axis(cfg->grid_w, cfg->tiles_x, cfg->resolution, cfg->x_min);
        AxisHost ay = build_axis(cfg->grid_h, cfg->tiles_y, cfg->resolution, cfg->y_min);
        m->tile_w = (double)cfg->grid_w * (double)cfg->resolution / cfg->tiles_x;
        m->tile_h = (double)cfg->grid_h * (double)cfg->resolution / cfg->tiles_y;
        if ((rc = upload(&m->bnd_x_lo, ax.bnd_lo)) || (rc = upload(&m->bnd_y_lo, ay.bnd_lo)) ||
            (rc = upload(&m->centre_x, centre_pairs(ax.centre))) ||
            (rc = upload(&m->centre_y, centre_pairs(ay.centre))) ||
            (rc = upload(&m->col_tile, ax.cell_tile)) || (rc = upload(&m->row_tile, ay.cell_tile)) ||
            (rc = upload(&m->col_off, ax.cell_off)) || (rc = upload(&m->row_off, ay.cell_off)))
            break;
        // Bundling patches.  Coarse: every patch's points lie within 30 / nu_max
        // of its centre (phases below 32 turns: the fast reduction).  Fine:
        // within 3.9 / nu_max (below 4 turns: MUFU sin/cos on unreduced phases).
        // At most 4096 segments each; beyond that, patches are larger and their
        // chunks take the next path.
        for (int level = 0; level < 2 && rc == VSAOGM_OK; ++level) {
            const double reach = level == 0 ? 60.0 : 7.8;  // patch width x nu_max
            int pnx = std::max(1, (int)std::ceil(m->tile_w * m->nu_max[0] / reach));
            int pny = std::max(1, (int)std::ceil(m->tile_h * m->nu_max[1] / reach));
            if (const char *v = getenv("VSAOGM_ENCODE_PATCHES"))
                if (atoi(v) == 0) pnx = pny = 1;
            while ((long long)m->S * pnx * pny > 4096 && (pnx > 1 || pny > 1)) {
                if (pnx >= pny) --pnx; else --pny;
            }
            std::vector<float> cxs(pnx), cys(pny);
            for (int p = 0; p < pnx; ++p) cxs[p] = (float)(-0.5 * m->tile_w + (p + 0.5) * m->tile_w / pnx);
            for (int p = 0; p < pny; ++p) cys[p] = (float)(-0.5 * m->tile_h + (p + 0.5) * m->tile_h / pny);
            if ((rc = upload(&m->patch_cx[level], cxs)) || (rc = upload(&m->patch_cy[level], cys)))
                break;
            PatchDev &pt = m->patches[level];
            pt.nx = pnx;
            pt.ny = pny;
            pt.n = pnx * pny;
            pt.hw_x = (float)(0.5 * m->tile_w);
            pt.hw_y = (float)(0.5 * m->tile_h);
            pt.inv_pw_x = (float)(pnx / m->tile_w);
            pt.inv_pw_y = (float)(pny / m->tile_h);
            pt.cx = m->patch_cx[level];
            pt.cy = m->patch_cy[level];
        }
        if (rc != VSAOGM_OK) break;
        // cells of each tile per axis; decode blocks are cut from these per call
        m->tile_first[0] = ax.first;
        m->tile_last[0] = ax.last;
        m->tile_first[1] = ay.first;
        m->tile_last[1] = ay.last;
        const std::vector<int> status0(1, 0);
        if ((rc = upload(&m->status, status0))) break;
        disk_half_widths(cfg->r_emp, m->r_hw[0]);
        disk_half_widths(cfg->r_occ, m->r_hw[1]);
        // Memories and per-map device state.
        cudaError_t e = dev_malloc((void **)&m->omega, sizeof(float2) * (size_t)m->S * D);
        if (e == cudaSuccess) e = dev_malloc((void **)&m->inv_norm, sizeof(float) * m->S);
        if (e == cudaSuccess) e = dev_malloc((void **)&m->maxima, sizeof(unsigned) * 2);
        if (e == cudaSuccess) e = dev_malloc((void **)&m->rejected, sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemset(m->omega, 0, sizeof(float2) * (size_t)m->S * D);
        if (e == cudaSuccess) e = cudaMemset(m->rejected, 0, sizeof(unsigned long long));
        // the encode's finished-chunk counters: one per memory and slice of at
        // least 512 frequencies; each is back at zero when a launch ends
        const size_t n_cnt = (size_t)m->S * ((D + 511) / 512);
        if (e == cudaSuccess) e = dev_malloc((void **)&m->enc_cnt, sizeof(unsigned) * n_cnt);
        if (e == cudaSuccess) e = cudaMemset(m->enc_cnt, 0, sizeof(unsigned) * n_cnt);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            rc = cuda_error(e, "map allocation");
            break;
        }
        if (cfg->decode_prec != VSAOGM_DECODE_FP32 && (rc = build_tc_tables(m))) break;
        // set-up of vsaogm_encode_bundle_noalloc on this device (the address
        // of its static scratch), so that its first call does no lookup
        unsigned char *scratch = nullptr;
        if ((rc = noalloc_scratch(m->device, &scratch))) break;
    } while (0);
    if (rc != VSAOGM_OK) {
        free_map(m);
        return rc;
    }
    *out = m;
    g_err[0] = 0;
    return VSAOGM_OK;
}

int vsaogm_destroy(vsaogm_map *m)
{
    if (!m) return VSAOGM_OK;
    cudaError_t e = cudaDeviceSynchronize();
    free_map(m);
    if (e != cudaSuccess) return cuda_error(e, "destroy");
    return VSAOGM_OK;
}

int vsaogm_reset(vsaogm_map *m, void *stream)
{
    if (!m) return set_error(VSAOGM_E_INVAL, "map is NULL");
    ++m->mem_gen;
    cudaStream_t st = (cudaStream_t)stream;
    VSA_CUDA(cudaMemsetAsync(m->omega, 0, sizeof(float2) * (size_t)m->S * m->cfg.D, st), "reset");
    VSA_CUDA(cudaMemsetAsync(m->rejected, 0, sizeof(unsigned long long), st), "reset");
    return VSAOGM_OK;
}

int vsaogm_encode_bundle(vsaogm_map *m, const float *xy, const uint8_t *lab, int64_t n,
                         void *stream)
{
    alloc_scope_begin();
    if (!m) return set_error(VSAOGM_E_INVAL, "map is NULL");
    ++m->mem_gen;
    if (n < 0) return set_error(VSAOGM_E_INVAL, "n must be >= 0");
    if (n == 0) return VSAOGM_OK;
    if (!xy || !lab) return set_error(VSAOGM_E_INVAL, "xy and labels must not be NULL");
    if ((uintptr_t)xy % 8 != 0) return set_error(VSAOGM_E_INVAL, "xy must be 8-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long before = 0;
    if (m->cfg.flags & VSAOGM_FLAG_CHECKED) {
        VSA_CUDA(cudaMemcpyAsync(&before, m->rejected, 8, cudaMemcpyDeviceToHost, st), "encode");
    }
    for (int64_t off = 0; off < n; off += kMaxBatch) {
        int64_t cnt = std::min<int64_t>(kMaxBatch, n - off);
        VSA_TRY(encode_bundle(m, xy + 2 * off, lab + off, cnt, st));
    }
    if (m->cfg.flags & VSAOGM_FLAG_CHECKED) {
        unsigned long long after = 0;
        VSA_CUDA(cudaMemcpyAsync(&after, m->rejected, 8, cudaMemcpyDeviceToHost, st), "encode");
        VSA_CUDA(cudaStreamSynchronize(st), "encode");
        if (after != before)
            return set_error(VSAOGM_E_DATA, "%llu points rejected (label > 1 or non-finite)",
                             after - before);
    }
    return VSAOGM_OK;
}

int vsaogm_decode(vsaogm_map *m, float *heat, void *stream)
{
    alloc_scope_begin();
    if (!m || !heat) return set_error(VSAOGM_E_INVAL, "map and heat must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    VSA_TRY(decode_raw(m, heat, st));
    return apply_nonlinearity(m, heat, st);
}

int vsaogm_entropy(vsaogm_map *m, const float *heat, float *occ, float *ogm, uint8_t *cls,
                   void *stream)
{
    alloc_scope_begin();
    if (!m || !heat || !occ) return set_error(VSAOGM_E_INVAL, "map, heat and occ must not be NULL");
    return entropy(m, heat, full_region(m), full_region(m), false, occ, ogm, cls,
                   (cudaStream_t)stream);
}

int vsaogm_query(vsaogm_map *m, float *heat, float *occ, float *ogm, uint8_t *cls, void *stream)
{
    alloc_scope_begin();
    if (!m || !heat || !occ) return set_error(VSAOGM_E_INVAL, "map, heat and occ must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    VSA_TRY(decode_raw(m, heat, st));
    return entropy(m, heat, full_region(m), full_region(m), true, occ, ogm, cls, st);
}

int vsaogm_window_scratch(const vsaogm_map *m, int32_t x0, int32_t y0, int32_t w, int32_t h,
                          int64_t *floats)
{
    if (!m || !floats) return set_error(VSAOGM_E_INVAL, "map and floats must not be NULL");
    if (w < 1 || h < 1 || x0 < 0 || y0 < 0 || x0 + w > m->cfg.grid_w || y0 + h > m->cfg.grid_h)
        return set_error(VSAOGM_E_INVAL, "window must lie inside the map");
    const int R = std::max(m->cfg.r_occ, m->cfg.r_emp);
    const int64_t rw = std::min(m->cfg.grid_w, x0 + w + R) - std::max(0, x0 - R);
    const int64_t rh = std::min(m->cfg.grid_h, y0 + h + R) - std::max(0, y0 - R);
    *floats = 2 * rw * rh;
    return VSAOGM_OK;
}

int vsaogm_query_window(vsaogm_map *m, int32_t x0, int32_t y0, int32_t w, int32_t h, float *heat,
                        float *occ, float *ogm, uint8_t *cls, void *stream)
{
    alloc_scope_begin();
    int64_t need;
    VSA_TRY(vsaogm_window_scratch(m, x0, y0, w, h, &need));
    if (!heat || !occ) return set_error(VSAOGM_E_INVAL, "heat and occ must not be NULL");
    const int R = std::max(m->cfg.r_occ, m->cfg.r_emp);
    const Region win{x0, y0, x0 + w, y0 + h};
    const Region r{std::max(0, x0 - R), std::max(0, y0 - R), std::min(m->cfg.grid_w, x0 + w + R),
                   std::min(m->cfg.grid_h, y0 + h + R)};
    cudaStream_t st = (cudaStream_t)stream;
    if (!(m->cfg.flags & VSAOGM_FLAG_WINDOW_MAP_MAX)) {
        VSA_TRY(decode_region(m, r, heat, st));
        return entropy(m, heat, r, win, true, occ, ogm, cls, st);
    }
    // the whole map's P and maxima (Eq. non-linearities over the map), decoded
    // again only when the memories have changed since
    const size_t W = m->cfg.grid_w, H = m->cfg.grid_h;
    VSA_TRY(ensure(m->ws.map_heat, sizeof(float) * 2 * W * H));
    float *mh = (float *)m->ws.map_heat.ptr;
    if (m->map_heat_gen != m->mem_gen) {
        m->map_heat_gen = ~0ull;
        VSA_TRY(decode_raw(m, mh, st));
        m->map_heat_gen = m->mem_gen;
    }
    for (int c = 0; c < 2; ++c)
        VSA_CUDA(cudaMemcpy2DAsync(heat + (size_t)c * r.w() * r.h(), sizeof(float) * r.w(),
                                   mh + c * W * H + (size_t)r.y0 * W + r.x0, sizeof(float) * W,
                                   sizeof(float) * r.w(), r.h(), cudaMemcpyDeviceToDevice, st),
                 "query_window");
    return entropy(m, mh, full_region(m), win, true, occ, ogm, cls, st);
}

int vsaogm_decode_window(vsaogm_map *m, int32_t x0, int32_t y0, int32_t w, int32_t h,
                         float *heat, void *stream)
{
    alloc_scope_begin();
    int64_t need;
    VSA_TRY(vsaogm_window_scratch(m, x0, y0, w, h, &need));
    if (!heat) return set_error(VSAOGM_E_INVAL, "heat must not be NULL");
    const Region win{x0, y0, x0 + w, y0 + h};
    const size_t cells = (size_t)w * h;
    cudaStream_t st = (cudaStream_t)stream;
    if (!(m->cfg.flags & VSAOGM_FLAG_WINDOW_MAP_MAX)) {
        // P of the window, its per-class maxima, then the non-linearity by them
        VSA_TRY(decode_region(m, win, heat, st));
        return apply_nonlinearity(m, heat, st, cells);
    }
    // the whole map's P and maxima, decoded again only when the memories have
    // changed since; the window's cells are copied out and normalised by the
    // map's maxima
    const size_t W = m->cfg.grid_w, H = m->cfg.grid_h;
    VSA_TRY(ensure(m->ws.map_heat, sizeof(float) * 2 * W * H));
    float *mh = (float *)m->ws.map_heat.ptr;
    if (m->map_heat_gen != m->mem_gen) {
        m->map_heat_gen = ~0ull;
        VSA_TRY(decode_raw(m, mh, st));
        m->map_heat_gen = m->mem_gen;
    }
    for (int c = 0; c < 2; ++c)
        VSA_CUDA(cudaMemcpy2DAsync(heat + (size_t)c * cells, sizeof(float) * w,
                                   mh + c * W * H + (size_t)y0 * W + x0, sizeof(float) * W,
                                   sizeof(float) * w, h, cudaMemcpyDeviceToDevice, st),
                 "decode_window");
    return apply_nonlinearity(m, heat, st, cells);
}

int vsaogm_update_query_host(vsaogm_map *m, const float *xy_host, const uint8_t *lab_host,
                             int64_t n, float *occ_host, void *stream)
{
    alloc_scope_begin();
    if (!m || !occ_host) return set_error(VSAOGM_E_INVAL, "map and occ_host must not be NULL");
    if (n < 0 || (n > 0 && (!xy_host || !lab_host)))
        return set_error(VSAOGM_E_INVAL, "bad point arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cells = (size_t)m->cfg.grid_w * m->cfg.grid_h;
    VSA_TRY(ensure(m->ws.stage_heat, sizeof(float) * 2 * cells));
    VSA_TRY(ensure(m->ws.stage_occ, sizeof(float) * cells));
    if (n > 0) {
        VSA_TRY(ensure(m->ws.stage_xy, sizeof(float) * 2 * (size_t)n));
        VSA_TRY(ensure(m->ws.stage_lab, (size_t)n));
        VSA_CUDA(cudaMemcpyAsync(m->ws.stage_xy.ptr, xy_host, sizeof(float) * 2 * (size_t)n,
                                 cudaMemcpyHostToDevice, st), "points upload");
        VSA_CUDA(cudaMemcpyAsync(m->ws.stage_lab.ptr, lab_host, (size_t)n, cudaMemcpyHostToDevice,
                                 st), "labels upload");
        VSA_TRY(vsaogm_encode_bundle(m, (const float *)m->ws.stage_xy.ptr,
                                     (const uint8_t *)m->ws.stage_lab.ptr, n, stream));
    }
    VSA_TRY(vsaogm_query(m, (float *)m->ws.stage_heat.ptr, (float *)m->ws.stage_occ.ptr, nullptr,
                         nullptr, stream));
    VSA_CUDA(cudaMemcpyAsync(occ_host, m->ws.stage_occ.ptr, sizeof(float) * cells,
                             cudaMemcpyDeviceToHost, st), "occupancy download");
    VSA_CUDA(cudaStreamSynchronize(st), "update_query_host");
    return VSAOGM_OK;
}

int vsaogm_reserve(vsaogm_map *m, int64_t max_points)
{
    alloc_scope_begin();
    if (!m) return set_error(VSAOGM_E_INVAL, "map is NULL");
    if (max_points < 0) return set_error(VSAOGM_E_INVAL, "max_points must be >= 0");
    VSA_TRY(reserve_encode(m, max_points));
    VSA_TRY(reserve_decode(m));
    if (m->cfg.flags & VSAOGM_FLAG_WINDOW_MAP_MAX)
        VSA_TRY(ensure(m->ws.map_heat,
                       sizeof(float) * 2 * (size_t)m->cfg.grid_w * m->cfg.grid_h));
    VSA_CUDA(cudaDeviceSynchronize(), "reserve");
    return VSAOGM_OK;
}

int vsaogm_rejected(vsaogm_map *m, int64_t *count, void *stream)
{
    if (!m || !count) return set_error(VSAOGM_E_INVAL, "map and count must not be NULL");
    unsigned long long v = 0;
    cudaStream_t st = (cudaStream_t)stream;
    VSA_CUDA(cudaMemcpyAsync(&v, m->rejected, 8, cudaMemcpyDeviceToHost, st), "rejected");
    VSA_CUDA(cudaStreamSynchronize(st), "rejected");
    *count = (int64_t)v;
    return VSAOGM_OK;
}

int vsaogm_get_memory(const vsaogm_map *m, float *omega, void *stream)
{
    if (!m || !omega) return set_error(VSAOGM_E_INVAL, "map and omega must not be NULL");
    VSA_CUDA(cudaMemcpyAsync(omega, m->omega, sizeof(float2) * (size_t)m->S * m->cfg.D,
                             cudaMemcpyDeviceToDevice, (cudaStream_t)stream), "get_memory");
    return VSAOGM_OK;
}

int vsaogm_set_memory(vsaogm_map *m, const float *omega, void *stream)
{
    if (!m || !omega) return set_error(VSAOGM_E_INVAL, "map and omega must not be NULL");
    ++m->mem_gen;
    VSA_CUDA(cudaMemcpyAsync(m->omega, omega, sizeof(float2) * (size_t)m->S * m->cfg.D,
                             cudaMemcpyDeviceToDevice, (cudaStream_t)stream), "set_memory");
    return VSAOGM_OK;
}

int vsaogm_fuse(vsaogm_map *dst, const vsaogm_map *src, void *stream)
{
    if (!dst || !src) return set_error(VSAOGM_E_INVAL, "maps must not be NULL");
    const vsaogm_config &a = dst->cfg, &b = src->cfg;
    // Algorithm 3's conditions: same axis vectors, same classes, same tiling.
    if (a.D != b.D || a.seed != b.seed || a.length_scale != b.length_scale ||
        a.tiles_x != b.tiles_x || a.tiles_y != b.tiles_y || a.grid_w != b.grid_w ||
        a.grid_h != b.grid_h || a.resolution != b.resolution || a.x_min != b.x_min ||
        a.y_min != b.y_min)
        return set_error(VSAOGM_E_INVAL,
                         "fusion needs the same axis vectors (D, seed, l) and the same tiling");
    if (dst->device != src->device) return set_error(VSAOGM_E_INVAL, "maps on different devices");
    if (dst == src) return set_error(VSAOGM_E_INVAL, "cannot fuse a map into itself");
    ++dst->mem_gen;
    return add_memories(dst->omega, src->omega, (int64_t)dst->S * a.D, (cudaStream_t)stream);
}

int vsaogm_get_axis_frequencies(const vsaogm_map *m, float *nu_x, float *nu_y)
{
    if (!m || !nu_x || !nu_y) return set_error(VSAOGM_E_INVAL, "NULL argument");
    memcpy(nu_x, m->host_nu, sizeof(float) * m->cfg.D);
    memcpy(nu_y, m->host_nu + m->cfg.D, sizeof(float) * m->cfg.D);
    return VSAOGM_OK;
}

int vsaogm_status(vsaogm_map *m, void *stream)
{
    if (!m) return set_error(VSAOGM_E_INVAL, "map is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int code = 0;
    VSA_CUDA(cudaMemcpyAsync(&code, m->status, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    VSA_CUDA(cudaStreamSynchronize(st), "status");
    if (code != 0) {
        VSA_CUDA(cudaMemset(m->status, 0, sizeof(int)), "status");
        if (code == VSAOGM_E_INVAL)
            return set_error(code, "the tensor-core decode refused an ill-formed block");
        return set_error(code, "a kernel gave up on a bounded wait (tensor-core decode)");
    }
    // the checked build's bounds records (always 0 in the normal build)
    const struct {
        const char *tu;
        int line;
    } checks[] = {{"encode.cu", take_check_line_encode()},
                  {"decode.cu", take_check_line_decode()},
                  {"decode_tc.cu", take_check_line_decode_tc()},
                  {"entropy.cu", take_check_line_entropy()}};
    for (const auto &c : checks)
        if (c.line != 0)
            return set_error(VSAOGM_E_DATA, "checked build: index out of range at %s:%d (access skipped)",
                             c.tu, c.line);
    return VSAOGM_OK;
}

int vsaogm_set_timing(vsaogm_map *m, int enable)
{
    if (!m) return set_error(VSAOGM_E_INVAL, "map is NULL");
    m->timer.enabled = enable != 0;
    return VSAOGM_OK;
}

int vsaogm_stage_times(vsaogm_map *m, double *ms, int64_t *launches, int reset)
{
    if (!m) return set_error(VSAOGM_E_INVAL, "map is NULL");
    StageTimer &t = m->timer;
    for (auto &p : t.pending) {
        cudaError_t e = cudaEventSynchronize(p.b);
        float dt = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&dt, p.a, p.b);
        if (e != cudaSuccess) return cuda_error(e, "stage_times");
        t.ms[p.stage] += dt;
        t.free_events.push_back(p.a);
        t.free_events.push_back(p.b);
    }
    t.pending.clear();
    for (int s = 0; s < VSAOGM_N_STAGES; ++s) {
        if (ms) ms[s] = t.ms[s];
        if (launches) launches[s] = t.launches[s];
        if (reset) {
            t.ms[s] = 0.0;
            t.launches[s] = 0;
        }
    }
    return VSAOGM_OK;
}

int vsaogm_get_shape(const vsaogm_map *m, int32_t *n_tiles, int32_t *n_memories)
{
    if (!m) return set_error(VSAOGM_E_INVAL, "map is NULL");
    if (n_tiles) *n_tiles = m->T;
    if (n_memories) *n_memories = m->S;
    return VSAOGM_OK;
}

}  // extern "C"
