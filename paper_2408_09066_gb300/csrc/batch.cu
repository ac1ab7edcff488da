// Many maps processed together (a batch): one step encodes and bundles one
// point set per map and queries every map, with one launch per stage across
// all maps, optionally captured once in a CUDA graph and replayed.
//
// Stages of a step:
//   reset (optional)  : memset of each map's memories
//   sort              : tile assignment + counting sort of every map, four
//                       launches (count, scan, chunk table, scatter), plus
//                       one launch sorting each small map in one CTA
//   encode            : ONE persistent launch over every map's (chunk,
//                       frequency slice) items, claimed from an atomic counter;
//                       for maps with few chunks per memory the last CTA of
//                       each (memory, slice) adds the memory's chunk partials
//                       in chunk order (fixed-order sums)
//   reduce            : ONE launch, the same sums for the other maps
//   norms             : ONE launch over every memory
//   decode            : ONE tensor-core launch over every map's (block, slice)
//   slice sums + max  : ONE launch (plus one tiny launch zeroing the maxima)
//   entropy           : ONE launch over every map's cells
// The shapes (share of polynomial phasors in the encode, chunk size, decode
// slicing) come from vsaogm_batch_autotune, which times candidates on the
// caller's own data and keeps the fastest.
#include <algorithm>
#include <array>
#include <cstring>
#include <vector>

#include "internal.cuh"

static_assert(vsaogm_impl::kMaxBatchMaps == VSAOGM_MAX_BATCH, "batch size limit");


using namespace vsaogm_impl;

namespace {

struct Tuning {
    int poly_warps = 9;       // polynomial pairs per CTA (warp w takes (w < p) + (w < p - 8)),
                              // for maps whose phases stay below 4 turns (2 fewer otherwise)
    int fine_min = 512;       // points per segment that warrant the fine bundling patches
    int items_per_cta = 8;    // encode work items per persistent CTA (sets the chunk size)
    int decode_waves = 2;     // decode items per SM
};
}  // namespace

struct vsaogm_batch {
    std::vector<vsaogm_map *> maps;
    std::vector<Scratch> ws;                    // per map: sort, partials and decode slices
    int decode_prec = VSAOGM_DECODE_BF16X3;     // shared by every map of the batch
    Tuning tune;
    int enc_ctas = 0;
    unsigned long long *counter = nullptr;      // encode work counter (device)
    BatchDecodeItem *items = nullptr;           // decode work list (device)
    int n_items = 0, items_cap = 0;
    int decode_waves_built = -1;
    std::vector<int> splits;                    // decode slices per map
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long graph_launches[VSAOGM_N_STAGES] = {};  // kernels of the captured step
    // stage timing: 7 events per timed step bound the stages sort (with the
    // reset), encode (with fused chunk sums), reduce (the other maps' chunk
    // sums), norms, decode (with the slice sums) and entropy
    bool timing = false;
    std::vector<cudaEvent_t> free_events;
    std::vector<std::array<cudaEvent_t, 7>> pending;
    double ms[VSAOGM_N_STAGES] = {};
    long long launches[VSAOGM_N_STAGES] = {};
};

namespace {

int batch_error(int code, const char *msg) { return set_error(code, "%s", msg); }

// Decode work list for the current slicing: every map's 128 x 128 blocks x its
// slices.  Rebuilt only when the slicing changes.
int build_decode_items(vsaogm_batch *b)
{
    if (b->decode_waves_built == b->tune.decode_waves) return VSAOGM_OK;
    std::vector<std::vector<DecodeBlock>> blocks(b->maps.size());
    size_t n_blocks = 0;
    for (size_t i = 0; i < b->maps.size(); ++i) {
        tc_blocks(b->maps[i], full_region(b->maps[i]), blocks[i]);
        n_blocks += blocks[i].size();
    }
    const int target = 152 * b->tune.decode_waves;
    const int s_all = std::max<int>(1, (int)((target + n_blocks - 1) / n_blocks));
    std::vector<BatchDecodeItem> items;
    b->splits.assign(b->maps.size(), 1);
    for (size_t i = 0; i < b->maps.size(); ++i) {
        vsaogm_map *m = b->maps[i];
        const int D = m->cfg.D;
        const int KS = tc_stage_freqs(b->decode_prec);
        int s = std::max((D + kTcMaxKPerSplit - 1) / kTcMaxKPerSplit,
                         std::min(s_all, (D + KS - 1) / KS));
        const int kps = ((D + s - 1) / s + KS - 1) / KS * KS;
        s = (D + kps - 1) / kps;
        b->splits[i] = s;
        for (const DecodeBlock &blk : blocks[i])
            for (int sp = 0; sp < s; ++sp) items.push_back(BatchDecodeItem{(int)i, sp, blk});
        const size_t cells = (size_t)m->cfg.grid_w * m->cfg.grid_h;
        int rc = ensure(b->ws[i].dec_partial, sizeof(float) * (size_t)s * 2 * cells);
        if (rc) return rc;
    }
    if ((int)items.size() > b->items_cap) {
        if (b->items) dev_free(b->items);
        b->items = nullptr;
        cudaError_t e = dev_malloc((void **)&b->items, sizeof(BatchDecodeItem) * items.size());
        if (e != cudaSuccess) return cuda_error(e, "batch decode items");
        b->items_cap = (int)items.size();
    }
    cudaError_t e = cudaMemcpy(b->items, items.data(), sizeof(BatchDecodeItem) * items.size(),
                               cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "batch decode items");
    b->n_items = (int)items.size();
    b->decode_waves_built = b->tune.decode_waves;
    return VSAOGM_OK;
}

// Points per encode chunk for this step (one size for every map).
int batch_chunk(const vsaogm_batch *b, const int64_t *n)
{
    double work = 0.0;
    for (size_t i = 0; i < b->maps.size(); ++i)
        work += (double)n[i] * ((b->maps[i]->cfg.D + 2047) / 2048);
    const double per_item = work / std::max(1.0, (double)b->enc_ctas * b->tune.items_per_cta);
    int c = 64;
    while (c * 2 <= per_item && c * 2 <= kMaxChunk) c *= 2;
    return c;
}

cudaEvent_t take_event(vsaogm_batch *b)
{
    if (!b->free_events.empty()) {
        cudaEvent_t e = b->free_events.back();
        b->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

constexpr int kStageOfMark[6] = {VSAOGM_STAGE_SORT,  VSAOGM_STAGE_ENCODE, VSAOGM_STAGE_REDUCE,
                                 VSAOGM_STAGE_NORMS, VSAOGM_STAGE_DECODE, VSAOGM_STAGE_ENTROPY};

// Enqueues one step; records the 7 stage-boundary events `ev` when non-NULL.
// `counted[stage]` receives the kernels it launches.
int enqueue_step(vsaogm_batch *b, const float *const *xy, const uint8_t *const *lab,
                 const int64_t *n, float *const *heat, float *const *occ, float *const *ogm,
                 int reset, cudaStream_t st, const std::array<cudaEvent_t, 7> *ev,
                 long long *counted)
{
    const int M = (int)b->maps.size();
    cudaError_t e;
    int rc;
    int mark_no = 0;
    auto mark = [&]() {
        if (ev) cudaEventRecord((*ev)[mark_no], st);
        ++mark_no;
    };
    for (int s = 0; s < VSAOGM_N_STAGES; ++s) counted[s] = 0;
    mark();
    if (reset)
        for (vsaogm_map *m : b->maps)
            if ((e = cudaMemsetAsync(m->omega, 0, sizeof(float2) * (size_t)m->S * m->cfg.D, st)) !=
                cudaSuccess)
                return cuda_error(e, "batch reset");
    // ---- encode: the sorts of every map (four launches), then one launch
    const int chunk = batch_chunk(b, n);
    BatchSortTable sot, sos;  // maps sorted by the four kernels / in one CTA each
    memset(&sot, 0, sizeof(sot));
    memset(&sos, 0, sizeof(sos));
    int small_s1 = 0;
    BatchEncodeTable et;
    memset(&et, 0, sizeof(et));
    BatchReduceTable rt;
    memset(&rt, 0, sizeof(rt));
    long long items = 0;
    int sort_blocks = 0, sort_segs = 0, max_s1 = 0, red_segs = 0, d_max = 0;
    for (int i = 0; i < M; ++i) {
        vsaogm_map *m = b->maps[i];
        int max_chunks = 0;
        const PatchDev &pt = choose_patches(m, n[i], b->tune.fine_min);
        if (n[i] > 0) {
            const bool small = sort_small((int)n[i], m->S * pt.n + 1);
            BatchSortMap &sm = small ? sos.m[sos.n_maps++] : sot.m[sot.n_maps++];
            if ((rc = batch_sort_entry(m, b->ws[i], pt, xy[i], lab[i], (int)n[i], chunk, &sm,
                                       &max_chunks)))
                return rc;
            if (small) {
                small_s1 = std::max(small_s1, sm.S + 1);
            } else {
                sm.blk_begin = sort_blocks;
                sm.seg_begin = sort_segs;
                sort_blocks += sm.nb;
                sort_segs += sort_scan_ctas(sm.S + 1);
                max_s1 = std::max(max_s1, sm.S + 1);
            }
        }
        BatchEncodeMap &em = et.m[i];
        batch_encode_entry(m, b->ws[i], pt, &em);
        em.poly_warps = patches_near(m, pt) ? b->tune.poly_warps
                                            : std::max(0, b->tune.poly_warps - 2);
        em.item_begin = items;
        items += (long long)max_chunks * em.slices;
        if (n[i] == 0) em.slices = 1;  // no items: max_chunks = 0
        // Maps whose memories hold few chunks each sum them inside the encode
        // launch (the last CTA of a memory walks its chunks); maps with many
        // chunks per memory leave that to the separate reduction launch.
        if (n[i] > 0 && (n[i] + chunk - 1) / chunk > (int64_t)kFusedChunksPerMemory * m->S) {
            em.tail.cnt = nullptr;
            BatchReduceMap &rm = rt.m[rt.n_maps++];
            batch_reduce_entry(m, b->ws[i], pt, &rm);
            rm.seg_begin = red_segs;
            red_segs += m->S;
            d_max = std::max(d_max, m->cfg.D);
        }
    }
    if (sot.n_maps > 0) {
        if ((rc = launch_sort_batch(sot, sort_blocks, sort_segs, max_s1, st))) return rc;
        counted[VSAOGM_STAGE_SORT] += 4;
    }
    if (sos.n_maps > 0) {
        if ((rc = launch_sort_small_batch(sos, small_s1, st))) return rc;
        counted[VSAOGM_STAGE_SORT] += 1;
    }
    mark();
    et.n_maps = M;
    et.poly_warps = b->tune.poly_warps;
    et.total = items;
    if (items > 0) {
        if ((rc = launch_encode_batch(et, b->counter, b->enc_ctas, st))) return rc;
        counted[VSAOGM_STAGE_ENCODE] = 1;
    }
    mark();
    rt.total_segs = red_segs;
    if (rt.n_maps > 0) {
        if ((rc = launch_reduce_batch(rt, d_max, st))) return rc;
        counted[VSAOGM_STAGE_REDUCE] = 1;
    }
    mark();
    // ---- query: norms, decode, slice sums + maxima, entropy
    BatchNormTable nt;
    memset(&nt, 0, sizeof(nt));
    int mems = 0;
    for (int i = 0; i < M; ++i) {
        nt.m[i] = BatchNormMap{b->maps[i]->omega, b->maps[i]->inv_norm, b->maps[i]->cfg.D, mems};
        mems += b->maps[i]->S;
    }
    nt.n_maps = M;
    if ((rc = launch_norms_batch(nt, mems, st))) return rc;
    counted[VSAOGM_STAGE_NORMS] = 1;
    mark();
    if ((rc = build_decode_items(b))) return rc;
    BatchDecodeTable dt;
    memset(&dt, 0, sizeof(dt));
    BatchOutTable ot;
    memset(&ot, 0, sizeof(ot));
    int ent_blocks = 0, sum_blocks = 0;
    for (int i = 0; i < M; ++i) {
        vsaogm_map *m = b->maps[i];
        const int D = m->cfg.D, s = b->splits[i], KS = tc_stage_freqs(b->decode_prec);
        const int kps = ((D + s - 1) / s + KS - 1) / KS * KS;
        const float u = tc_u_scale(m);
        dt.m[i] = BatchDecodeMap{m->omega, m->inv_norm, m->nu, m->col_off, m->row_off,
                                 m->tc_rot, m->row_tile, (float *)b->ws[i].dec_partial.ptr,
                                 m->status, D, kps, m->cfg.grid_w, m->cfg.grid_h,
                                 m->cfg.tiles_x, u, m->debug_wait_ns, m->tc_xtmap};
        BatchMapOut &o = ot.m[i];
        o.partial = (const float *)b->ws[i].dec_partial.ptr;
        o.heat = heat[i];
        o.maxima = m->maxima;
        o.occ = occ[i];
        o.ogm = ogm ? ogm[i] : nullptr;
        o.splits = s;
        o.W = m->cfg.grid_w;
        o.H = m->cfg.grid_h;
        o.inv_scale = 1.0f / u;
        o.rho = m->cfg.rho;
        o.r[0] = m->cfg.r_emp;
        o.r[1] = m->cfg.r_occ;
        o.mode = m->cfg.decode_mode;
        o.blk_begin = ent_blocks;
        ent_blocks += ((o.W + 31) / 32) * ((o.H + 31) / 32);
        o.sum_begin = sum_blocks;
        sum_blocks += (int)((2 * (size_t)o.W * o.H + kSumBlockOutputs - 1) / kSumBlockOutputs);
    }
    dt.n_maps = ot.n_maps = M;
    if ((rc = launch_decode_tc_batch(dt, b->items, b->n_items, b->decode_prec, st))) return rc;
    if ((rc = launch_sums_batch(ot, sum_blocks, st))) return rc;
    counted[VSAOGM_STAGE_DECODE] = 3;
    mark();
    if ((rc = launch_entropy_batch(ot, st))) return rc;
    counted[VSAOGM_STAGE_ENTROPY] = 1;
    mark();
    return VSAOGM_OK;
}

// One step, timed per stage when the batch's timing is on (never while capturing).
int run_step(vsaogm_batch *b, const float *const *xy, const uint8_t *const *lab,
             const int64_t *n, float *const *heat, float *const *occ, float *const *ogm,
             int reset, cudaStream_t st, bool capturing = false)
{
    long long counted[VSAOGM_N_STAGES];
    std::array<cudaEvent_t, 7> ev{};
    const bool timed = b->timing && !capturing;
    if (timed)
        for (auto &x : ev)
            if (!(x = take_event(b))) {
                for (auto &y : ev)
                    if (y) b->free_events.push_back(y);
                return set_error(VSAOGM_E_CUDA, "batch timing: cudaEventCreate failed");
            }
    int rc = enqueue_step(b, xy, lab, n, heat, occ, ogm, reset, st, timed ? &ev : nullptr,
                          counted);
    if (timed) {
        if (rc == VSAOGM_OK)
            b->pending.push_back(ev);
        else
            for (auto &y : ev) b->free_events.push_back(y);
    }
    if (capturing)
        for (int s = 0; s < VSAOGM_N_STAGES; ++s) b->graph_launches[s] = counted[s];
    else if (rc == VSAOGM_OK)
        for (int s = 0; s < VSAOGM_N_STAGES; ++s) b->launches[s] += counted[s];
    return rc;
}

// Addresses of every buffer a step uses: a captured graph holds them, so a
// step that moves one (scratch that had to grow) invalidates the graph.
size_t scratch_signature(const vsaogm_batch *b)
{
    size_t h = (size_t)b->items;
    for (const Scratch &w : b->ws) {
        const DevBuf *bufs[] = {&w.blk_hist, &w.seg_meta, &w.chunks, &w.sorted, &w.partial,
                                &w.dec_partial};
        for (const DevBuf *d : bufs) h = h * 1000003u ^ (size_t)d->ptr;
    }
    return h;
}

void drop_graph(vsaogm_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// A step writes every map's memories (window queries that normalise by the
// whole map must decode it again).
void bump_generations(vsaogm_batch *b)
{
    for (vsaogm_map *m : b->maps) ++m->mem_gen;
}

}  // namespace

extern "C" {

int vsaogm_batch_create(vsaogm_map *const *maps, int32_t count, vsaogm_batch **out)
{
    alloc_scope_begin();
    if (!out || !maps) return set_error(VSAOGM_E_INVAL, "NULL argument");
    *out = nullptr;
    if (count < 1 || count > kMaxBatchMaps)
        return set_error(VSAOGM_E_INVAL, "a batch holds 1 to %d maps", kMaxBatchMaps);
    for (int i = 0; i < count; ++i) {
        if (!maps[i]) return batch_error(VSAOGM_E_INVAL, "NULL map in the batch");
        if (maps[i]->cfg.decode_prec == VSAOGM_DECODE_FP32)
            return batch_error(VSAOGM_E_INVAL, "batched decode runs on tensor cores: use "
                                               "VSAOGM_DECODE_BF16X3, FP16X3 or FP8X3");
        if (maps[i]->cfg.decode_prec != maps[0]->cfg.decode_prec)
            return batch_error(VSAOGM_E_INVAL, "all maps of a batch share decode_prec");
        if (maps[i]->device != maps[0]->device)
            return batch_error(VSAOGM_E_INVAL, "all maps of a batch share the device");
        if (maps[i]->cfg.flags & VSAOGM_FLAG_ATOMIC)
            return batch_error(VSAOGM_E_INVAL, "batched maps use the deterministic bundling");
        for (int j = 0; j < i; ++j)
            if (maps[j] == maps[i]) return batch_error(VSAOGM_E_INVAL, "a map appears twice");
    }
    vsaogm_batch *b = new (std::nothrow) vsaogm_batch();
    if (!b) return set_error(VSAOGM_E_NOMEM, "host allocation");
    b->maps.assign(maps, maps + count);
    b->ws.resize(count);
    b->decode_prec = maps[0]->cfg.decode_prec;
    b->enc_ctas = encode_batch_ctas();
    cudaError_t e = dev_malloc((void **)&b->counter, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        int rc = cuda_error(e, "batch create");
        vsaogm_batch_destroy(b);
        return rc;
    }
    *out = b;
    return VSAOGM_OK;
}

int vsaogm_batch_destroy(vsaogm_batch *b)
{
    if (!b) return VSAOGM_OK;
    cudaDeviceSynchronize();
    drop_graph(b);
    if (b->counter) dev_free(b->counter);
    if (b->items) dev_free(b->items);
    for (Scratch &w : b->ws) free_scratch(w);
    for (cudaEvent_t e : b->free_events) cudaEventDestroy(e);
    for (auto &p : b->pending)
        for (cudaEvent_t e : p) cudaEventDestroy(e);
    delete b;
    return VSAOGM_OK;
}

static int check_step_args(vsaogm_batch *b, const float *const *xy, const uint8_t *const *lab,
                           const int64_t *n, float *const *heat, float *const *occ)
{
    if (!b || !xy || !lab || !n || !heat || !occ) return set_error(VSAOGM_E_INVAL, "NULL argument");
    for (size_t i = 0; i < b->maps.size(); ++i) {
        if (n[i] < 0 || n[i] > kMaxBatch) return set_error(VSAOGM_E_INVAL, "bad point count");
        if (n[i] > 0 && (!xy[i] || !lab[i] || (uintptr_t)xy[i] % 8))
            return set_error(VSAOGM_E_INVAL, "bad point arrays for map %zu", i);
        if (!heat[i] || !occ[i]) return set_error(VSAOGM_E_INVAL, "NULL output for map %zu", i);
    }
    return VSAOGM_OK;
}

int vsaogm_batch_step(vsaogm_batch *b, const float *const *xy, const uint8_t *const *lab,
                      const int64_t *n, float *const *heat, float *const *occ,
                      float *const *ogm, int32_t reset, void *stream)
{
    alloc_scope_begin();
    int rc = check_step_args(b, xy, lab, n, heat, occ);
    if (rc) return rc;
    bump_generations(b);
    const size_t sig = scratch_signature(b);
    rc = run_step(b, xy, lab, n, heat, occ, ogm, reset, (cudaStream_t)stream);
    if (b->exec && scratch_signature(b) != sig) drop_graph(b);
    return rc;
}

int vsaogm_batch_capture(vsaogm_batch *b, const float *const *xy, const uint8_t *const *lab,
                         const int64_t *n, float *const *heat, float *const *occ,
                         float *const *ogm, int32_t reset, void *stream)
{
    alloc_scope_begin();
    int rc = check_step_args(b, xy, lab, n, heat, occ);
    if (rc) return rc;
    bump_generations(b);
    cudaStream_t st = (cudaStream_t)stream;
    if (!st) return set_error(VSAOGM_E_INVAL, "capture needs a non-default stream");
    for (vsaogm_map *m : b->maps)
        if (m->timer.enabled)
            return set_error(VSAOGM_E_INVAL, "turn stage timing off on batched maps to capture");
    // one uncaptured step grows every scratch buffer, so the captured one allocates nothing
    if ((rc = run_step(b, xy, lab, n, heat, occ, ogm, reset, st))) return rc;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "batch capture");
    drop_graph(b);
    if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_error(e, "batch capture");
    rc = run_step(b, xy, lab, n, heat, occ, ogm, reset, st, true);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(st, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_error(e, "batch capture");
    b->graph = g;
    if ((e = cudaGraphInstantiate(&b->exec, g, 0)) != cudaSuccess) {
        drop_graph(b);
        return cuda_error(e, "batch graph instantiate");
    }
    return VSAOGM_OK;
}

int vsaogm_batch_replay(vsaogm_batch *b, void *stream)
{
    if (!b) return set_error(VSAOGM_E_INVAL, "batch is NULL");
    if (!b->exec) return set_error(VSAOGM_E_INVAL, "no captured step: call vsaogm_batch_capture");
    bump_generations(b);
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_error(e, "batch replay");
    for (int s = 0; s < VSAOGM_N_STAGES; ++s) b->launches[s] += b->graph_launches[s];
    return VSAOGM_OK;
}

int vsaogm_batch_autotune(vsaogm_batch *b, const float *const *xy, const uint8_t *const *lab,
                          const int64_t *n, float *const *heat, float *const *occ, void *stream,
                          int32_t *poly_warps, int32_t *items_per_cta, int32_t *decode_waves)
{
    alloc_scope_begin();
    int rc = check_step_args(b, xy, lab, n, heat, occ);
    if (rc) return rc;
    bump_generations(b);
    drop_graph(b);  // the candidates grow and move the scratch a captured step uses
    const bool timing = b->timing;
    b->timing = false;  // candidates are timed here, not in the stage record
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    auto time_step = [&](float *ms) -> int {
        int r = run_step(b, xy, lab, n, heat, occ, nullptr, 1, st);  // warm (and grow scratch)
        if (r) return r;
        float best = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(t0, st);
            if ((r = run_step(b, xy, lab, n, heat, occ, nullptr, 1, st))) return r;
            cudaEventRecord(t1, st);
            cudaError_t e = cudaEventSynchronize(t1);
            if (e != cudaSuccess) return cuda_error(e, "autotune");
            float t = 0.f;
            cudaEventElapsedTime(&t, t0, t1);
            best = std::min(best, t);
        }
        *ms = best;
        return VSAOGM_OK;
    };
    Tuning best = b->tune;
    float best_ms = 1e30f;
    // encode shape first (decode fixed), then the decode slicing
    const int pws[] = {7, 8, 9, 10}, ipcs[] = {8, 16, 32};
    for (int pw : pws)
        for (int ipc : ipcs) {
            if (rc) break;
            b->tune.poly_warps = pw;
            b->tune.items_per_cta = ipc;
            float ms = 0.f;
            if ((rc = time_step(&ms))) break;
            if (ms < best_ms) {
                best_ms = ms;
                best = b->tune;
            }
        }
    b->tune = best;
    const int waves[] = {1, 2, 4};
    for (int w : waves) {
        if (rc) break;
        b->tune.decode_waves = w;
        float ms = 0.f;
        if ((rc = time_step(&ms))) break;
        if (ms < best_ms) {
            best_ms = ms;
            best = b->tune;
        }
    }
    b->tune = best;
    // how dense a map's points must be for the fine bundling patches
    const int fines[] = {16, 64, 128, 256, 1024, 2048};
    for (int f : fines) {
        if (rc) break;
        b->tune.fine_min = f;
        float ms = 0.f;
        if ((rc = time_step(&ms))) break;
        if (ms < best_ms) {
            best_ms = ms;
            best = b->tune;
        }
    }
    b->tune = best;
    b->timing = timing;
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (rc) return rc;
    if (poly_warps) *poly_warps = best.poly_warps;
    if (items_per_cta) *items_per_cta = best.items_per_cta;
    if (decode_waves) *decode_waves = best.decode_waves;
    return VSAOGM_OK;
}

int vsaogm_batch_set_timing(vsaogm_batch *b, int32_t enable)
{
    if (!b) return set_error(VSAOGM_E_INVAL, "batch is NULL");
    b->timing = enable != 0;
    return VSAOGM_OK;
}

int vsaogm_batch_stage_times(vsaogm_batch *b, double *ms, int64_t *launches, int32_t reset)
{
    if (!b) return set_error(VSAOGM_E_INVAL, "batch is NULL");
    for (auto &p : b->pending) {
        cudaError_t e = cudaEventSynchronize(p[6]);
        for (int k = 0; k < 6 && e == cudaSuccess; ++k) {
            float dt = 0.f;
            e = cudaEventElapsedTime(&dt, p[k], p[k + 1]);
            b->ms[kStageOfMark[k]] += dt;
        }
        if (e != cudaSuccess) return cuda_error(e, "batch stage times");
        for (cudaEvent_t x : p) b->free_events.push_back(x);
    }
    b->pending.clear();
    for (int s = 0; s < VSAOGM_N_STAGES; ++s) {
        if (ms) ms[s] = b->ms[s];
        if (launches) launches[s] = b->launches[s];
        if (reset) {
            b->ms[s] = 0.0;
            b->launches[s] = 0;
        }
    }
    return VSAOGM_OK;
}

}  // extern "C"
