// C ABI of the sDTW library (include/sdtw.h): contexts, argument checks,
// device workspace, launch plans and the autotuner, host-buffer entry points.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "sdtw.h"
#include "sdtw_internal.h"

using sdtw::FwdArgs;
using sdtw::FwdPlan;

namespace {

constexpr size_t kDefaultCap = size_t(16) << 30;
constexpr int64_t kMaxSmem = sdtw::kMaxSmemBytes;
constexpr int kI8MaxN = sdtw::kIntMaxN;
// steps between the checkpointing forward's wavefront stores when neither the
// caller nor the autotuner chose: 16-step bands (64 rows with 4-row tiles) make
// the backward's recompute per band change short
constexpr int kDefaultStride = 16;
// the strides the autotuner times for a context that keeps checkpoints
constexpr int kStrides[] = {8, 16, 32, 64};

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// shape class a tuned plan applies to
struct TuneKey {
    int dtype, ragged, nbucket, mbucket, ckpt;
    bool operator<(const TuneKey& o) const
    {
        return std::tie(dtype, ragged, nbucket, mbucket, ckpt) <
               std::tie(o.dtype, o.ragged, o.nbucket, o.mbucket, o.ckpt);
    }
};

int bucket_of(int64_t v)
{
    int b = 0;
    while (v > 1) {
        v >>= 1;
        ++b;
    }
    return b;
}

// the inputs and plan of the forward whose checkpoints the workspace holds
struct CkptKey {
    const void* ref = nullptr;
    const void* queries = nullptr;
    const int64_t* offsets = nullptr;
    int64_t M = 0;
    int32_t B = 0, N = 0;
    int32_t W = 0, P = 0, RT = 0, KS = 0;
    bool valid = false;
};

}  // namespace

struct sdtw_ctx {
    sdtw_config cfg{};
    int sm_count = 0;
    std::string err;
    size_t cap = kDefaultCap;
    size_t ws_bytes = 0;

    int* d_status = nullptr;
    int* d_queue = nullptr;
    int32_t* d_order = nullptr;

    // backward workspace: one arena, carved per call into the checkpoint
    // slots, gradient rows and per-query scalars of a chunk of queries
    float* d_arena = nullptr;
    size_t arena_floats = 0;
    void* d_cost_tmp = nullptr;
    int64_t* d_end_tmp = nullptr;
    CkptKey key;

    // host-call staging
    DevBuf st_ref, st_q, st_off, st_cost, st_end, st_gc, st_gq, st_gr, st_path;

    // SDTW_FLAG_ZNORM_QUERIES: the z-normalised queries (max_total_query_len floats)
    float* d_zq = nullptr;

    std::map<TuneKey, std::tuple<int, int, int, int>> tuned;  // -> (W, P, RT, checkpoint stride)
};

namespace {

sdtw_status cuda_fail(sdtw_ctx* c, cudaError_t e)
{
    if (c) c->err = cudaGetErrorString(e);
    return SDTW_E_CUDA;
}

size_t elem_size(sdtw_dtype dt) { return dt == SDTW_F32 ? 4 : dt == SDTW_F16 ? 2 : 1; }

bool int_mode(sdtw_dtype dt) { return dt == SDTW_I8 || dt == SDTW_U8; }

// CTAs of a non-persistent launch over nq queries (binary16 runs two queries per CTA)
int plain_grid(sdtw_dtype dt, int nq) { return dt == SDTW_F16 ? (nq + 1) / 2 : nq; }

sdtw_status dev_alloc(sdtw_ctx* c, void** p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) return SDTW_OK;
    if (c->ws_bytes + bytes > c->cap) return SDTW_E_NOMEM;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        c->err = cudaGetErrorString(e);
        return SDTW_E_NOMEM;
    }
    c->ws_bytes += bytes;
    return SDTW_OK;
}

void dev_free(sdtw_ctx* c, void* p, size_t bytes)
{
    if (p) {
        cudaFree(p);
        c->ws_bytes -= bytes;
    }
}

sdtw_status ensure(sdtw_ctx* c, DevBuf& b, size_t bytes)
{
    if (b.bytes >= bytes && (b.p || bytes == 0)) return SDTW_OK;
    dev_free(c, b.p, b.bytes);
    b.p = nullptr;
    b.bytes = 0;
    sdtw_status s = dev_alloc(c, &b.p, bytes);
    if (s == SDTW_OK) b.bytes = bytes;
    return s;
}

// default plan for a forward call
FwdPlan default_fwd_plan(const sdtw_ctx* c, int B, int N, int64_t M, bool ragged, bool ckpt)
{
    // defaults measured on the paper's batch: four warps per query; plain
    // fills with 8-row tiles of 24 columns (FP32, binary16) or 28 (the integer
    // modes; with pruning 4-row tiles, 22% faster there); the fill with
    // checkpoints with 4-row tiles of 28 columns and a checkpoint every 16
    // steps (fewer spills than 32 columns: a fill 0.6 ms faster, against
    // 0.2 ms more backward for its narrower windows; its 8-row plans, W 16
    // to 28, are the autotuner's to choose)
    FwdPlan p;
    p.W = c->cfg.seg_width > 0 ? c->cfg.seg_width : (ckpt || int_mode(c->cfg.dtype) ? 28 : 24);
    p.P = c->cfg.warps_per_query > 0 ? c->cfg.warps_per_query : 4;
    p.RT = c->cfg.tile_rows > 0 ? c->cfg.tile_rows
                                : (!ckpt && sdtw::fwd_plan_supported(c->cfg.dtype, p.W, 8, false) && c->cfg.prune_gap == 0
                                       ? 8
                                       : 4);
    // 64-row bands: 8 steps of 8-row tiles, 16 of 4-row tiles
    p.KS = c->cfg.ckpt_stride > 0 ? c->cfg.ckpt_stride : (p.RT == 8 ? 8 : kDefaultStride);
    auto it = c->tuned.find(TuneKey{c->cfg.dtype, ragged ? 1 : 0, bucket_of(N), bucket_of(M), ckpt ? 1 : 0});
    if (it != c->tuned.end()) {
        if (c->cfg.seg_width <= 0) p.W = std::get<0>(it->second);
        if (c->cfg.warps_per_query <= 0) p.P = std::get<1>(it->second);
        if (c->cfg.tile_rows <= 0) p.RT = std::get<2>(it->second);
        if (c->cfg.ckpt_stride <= 0) p.KS = std::get<3>(it->second);
    }
    // a short reference needs fewer threads per query (unless the caller fixed P)
    if (c->cfg.warps_per_query <= 0)
        while (p.P > 1 && static_cast<int64_t>(32) * (p.P / 2) * p.W >= M) p.P /= 2;
    p.block = 32 * p.P;
    p.smem = sdtw::fwd_smem_bytes(c->cfg.dtype, N, p.P, p.W, p.RT);
    p.persistent = ragged;
    if (p.persistent) {
        // 0 CTAs per SM when the query does not fit in shared memory: the call
        // then fails with SDTW_E_UNSUPPORTED before any launch
        const int per_sm = sdtw::fwd_max_ctas_per_sm(c->cfg.dtype, p.W, p.P, p.smem, p.RT, ckpt, c->cfg.prune_gap > 0);
        p.grid = std::max(1, std::min(B, per_sm * c->sm_count));
    } else {
        p.grid = plain_grid(c->cfg.dtype, B);
    }
    return p;
}

sdtw_status check_common(sdtw_ctx* c, const void* ref, int64_t M, const void* queries, int32_t B, int32_t N,
                         const void* o1, const void* o2)
{
    if (!c) return SDTW_E_INVALID;
    if (B < 0 || M < 1 || N < 1) return SDTW_E_INVALID;
    if (M > c->cfg.max_ref_len || N > c->cfg.max_query_len || B > c->cfg.max_batch) return SDTW_E_INVALID;
    if (M > INT_MAX / 2) return SDTW_E_INVALID;
    if (B > 0 && (!ref || !queries || !o1 || !o2)) return SDTW_E_INVALID;
    if (int_mode(c->cfg.dtype) && N > kI8MaxN) return SDTW_E_INVALID;
    return SDTW_OK;
}

// Backward workspace of a checkpointing plan, per query of a chunk (floats):
// the wavefront slot, the boundary columns, the reference-gradient row and
// the scalars (cost, end, span).
struct CkLayout {
    int64_t fr_slot = 0, ck_slot = 0, per_q = 0;
    int K = 0;
};

CkLayout ck_layout(int64_t M, int N, const FwdPlan& p)
{
    CkLayout l;
    l.K = 8 * p.W;
    l.fr_slot = sdtw::fr_slot_floats(M, N, p.W, p.P, p.RT, p.KS);
    l.ck_slot = sdtw::ck_slot_floats(M, N, l.K);
    l.per_q = l.fr_slot + l.ck_slot + M + 7;
    return l;
}

constexpr int64_t kCarveSlack = 32;  // rounding of the carved arrays to 16 bytes

// queries whose checkpoints fit in the arena at once
int64_t chunk_capacity(const sdtw_ctx* c, const CkLayout& l)
{
    if (c->arena_floats <= static_cast<size_t>(kCarveSlack)) return 0;
    return static_cast<int64_t>((c->arena_floats - kCarveSlack) / static_cast<size_t>(l.per_q));
}

// checkpoint arrays of a chunk of nq queries, carved from the arena
struct CkPtrs {
    float* fr = nullptr;
    int64_t fr_slot = 0;
    float* colck = nullptr;
    int64_t ck_slot = 0;
    int K = 0;
    float* gyq = nullptr;
    float* ck_cost = nullptr;
    int64_t* ck_end = nullptr;
    int64_t* span = nullptr;
};

CkPtrs carve(const sdtw_ctx* c, const CkLayout& l, int64_t nq, int64_t M)
{
    auto r4 = [](int64_t v) { return (v + 3) / 4 * 4; };
    CkPtrs k;
    k.fr_slot = l.fr_slot;
    k.ck_slot = l.ck_slot;
    k.K = l.K;
    k.fr = c->d_arena;
    k.colck = k.fr + nq * l.fr_slot;
    k.gyq = k.colck + r4(nq * l.ck_slot);
    k.ck_cost = k.gyq + r4(nq * M);
    k.ck_end = reinterpret_cast<int64_t*>(k.ck_cost + r4(nq));
    k.span = k.ck_end + r4(nq);
    return k;
}

sdtw_status run_forward(sdtw_ctx* c, const void* ref, int64_t M, const void* queries, const int64_t* offsets,
                        int32_t B, int32_t N, void* cost, int64_t* end, cudaStream_t s, const FwdPlan* force,
                        const CkPtrs* ck, int32_t q0, int32_t nq)
{
    const bool ragged = offsets != nullptr;
    FwdPlan p = force ? *force : default_fwd_plan(c, nq, N, M, ragged, ck != nullptr);
    if (p.smem > kMaxSmem) return SDTW_E_UNSUPPORTED;
    if (sdtw::fwd_total_steps(M, N, p.W, p.P, p.RT) > INT_MAX - 4 * sdtw::kChunk) return SDTW_E_UNSUPPORTED;
    if (p.persistent) p.grid = std::min(p.grid, nq);
    else p.grid = plain_grid(c->cfg.dtype, nq);
    FwdArgs a{};
    a.ref = ref;
    a.M = M;
    a.queries = queries;
    a.offsets = offsets;
    a.B = nq;
    a.N = N;
    a.q0 = q0;
    a.B_total = B;
    a.cost = cost;
    a.end = end;
    if (ck) {
        a.fr = ck->fr;
        a.fr_slot = ck->fr_slot;
        a.colck = ck->colck;
        a.ck_slot = ck->ck_slot;
        a.K = ck->K;
        a.ck_cost = ck->ck_cost;
        a.ck_end = ck->ck_end;
        a.ck_stride = p.KS;
        a.rebase_period = sdtw::ckpt_rebase_period(p.KS);
    } else {
        a.K = 1;
        a.ck_stride = sdtw::kChunk;
        // in a context that runs backwards, rebase like the checkpointing
        // fill of this shape: a forward then returns the same costs whether
        // or not it stores checkpoints
        a.rebase_period = (c->cfg.flags & SDTW_FLAG_GRAD) && c->cfg.dtype == SDTW_F32
                              ? sdtw::ckpt_rebase_period(default_fwd_plan(c, B, N, M, ragged, true).KS)
                              : sdtw::kChunk;
    }
    a.status = c->d_status;
    // the context's normalised copy holds max_total_query_len samples
    a.q_limit = (c->cfg.flags & SDTW_FLAG_ZNORM_QUERIES) ? c->cfg.max_total_query_len : 0;
    a.prune_gap = c->cfg.prune_gap;
    a.queue = nullptr;
    a.order = nullptr;
    cudaError_t e;
    if (p.persistent) {
        if ((e = cudaMemsetAsync(c->d_queue, 0, sizeof(int), s)) != cudaSuccess) return cuda_fail(c, e);
        if (ragged && q0 == 0 && nq == B) {
            if ((e = sdtw::launch_order_by_length(offsets, B, c->d_order, s)) != cudaSuccess) return cuda_fail(c, e);
            a.order = c->d_order;
        }
        a.queue = c->d_queue;
    }
    if ((e = sdtw::launch_forward(c->cfg.dtype, p, a, s)) != cudaSuccess) return cuda_fail(c, e);
    return SDTW_OK;
}

sdtw_status alloc_backward(sdtw_ctx* c)
{
    const sdtw_config& f = c->cfg;
    const int64_t M = f.max_ref_len;
    const int N = f.max_query_len;
    // one arena for the default checkpointing plan at the configured maxima:
    // the whole batch if the cap allows, else as many queries as fit (the
    // backward then runs in chunks of queries)
    const FwdPlan p = default_fwd_plan(c, f.max_batch, N, M, false, true);
    const CkLayout l = ck_layout(M, N, p);
    const size_t fixed = c->ws_bytes + 12 * static_cast<size_t>(f.max_batch);
    if (fixed + 4 * static_cast<size_t>(l.per_q + kCarveSlack) > c->cap) return SDTW_E_NOMEM;
    const size_t want = static_cast<size_t>(l.per_q) * f.max_batch + kCarveSlack;
    const size_t fit = (c->cap - fixed) / 4;
    c->arena_floats = std::min(want, fit);
    sdtw_status s;
    if ((s = dev_alloc(c, reinterpret_cast<void**>(&c->d_arena), 4 * c->arena_floats)) != SDTW_OK) return s;
    if ((s = dev_alloc(c, &c->d_cost_tmp, 4 * static_cast<size_t>(f.max_batch))) != SDTW_OK) return s;
    if ((s = dev_alloc(c, reinterpret_cast<void**>(&c->d_end_tmp), 8 * static_cast<size_t>(f.max_batch))) != SDTW_OK)
        return s;
    return SDTW_OK;
}

void free_all(sdtw_ctx* c)
{
    dev_free(c, c->d_status, sizeof(int));
    dev_free(c, c->d_queue, sizeof(int));
    dev_free(c, c->d_order, 4 * static_cast<size_t>(c->cfg.max_batch));
    dev_free(c, c->d_arena, 4 * c->arena_floats);
    dev_free(c, c->d_cost_tmp, 4 * static_cast<size_t>(c->cfg.max_batch));
    dev_free(c, c->d_end_tmp, 8 * static_cast<size_t>(c->cfg.max_batch));
    dev_free(c, c->d_zq, 4 * static_cast<size_t>(c->cfg.max_total_query_len));
    for (DevBuf* b : {&c->st_ref, &c->st_q, &c->st_off, &c->st_cost, &c->st_end, &c->st_gc, &c->st_gq, &c->st_gr,
                      &c->st_path})
        dev_free(c, b->p, b->bytes);
}

// The queries the fill reads: the caller's, or with SDTW_FLAG_ZNORM_QUERIES
// their z-normalised copy in the context (written here, on the stream).
sdtw_status fill_queries(sdtw_ctx* c, const void* queries, const int64_t* offsets, int32_t B, int32_t N, cudaStream_t st,
                         const void** out)
{
    *out = queries;
    if (!(c->cfg.flags & SDTW_FLAG_ZNORM_QUERIES) || B == 0) return SDTW_OK;
    const cudaError_t e = sdtw::launch_znormalize(static_cast<const float*>(queries), c->d_zq, offsets, B, N,
                                                  c->cfg.max_total_query_len, c->d_status, st);
    if (e != cudaSuccess) return cuda_fail(c, e);
    *out = c->d_zq;
    return SDTW_OK;
}

bool key_matches(const CkptKey& k, const void* ref, int64_t M, const void* q, const int64_t* off, int32_t B,
                 int32_t N)
{
    return k.valid && k.ref == ref && k.M == M && k.queries == q && k.offsets == off && k.B == B && k.N == N;
}

// the plan a checkpointing forward of this shape runs, and whether the whole
// batch's checkpoints fit in the arena
FwdPlan ckpt_plan(const sdtw_ctx* c, int32_t B, int32_t N, int64_t M, bool ragged)
{
    return default_fwd_plan(c, B, N, M, ragged, true);
}

bool keep_fits(const sdtw_ctx* c, int32_t B, int32_t N, int64_t M, const FwdPlan& p)
{
    return (c->cfg.flags & SDTW_FLAG_KEEP_CHECKPOINTS) && B <= chunk_capacity(c, ck_layout(M, N, p));
}

}  // namespace

// A profiler range (NVTX) over one call of the library, so that a timeline
// tool attributes the call's launches; without a tool attached it costs a
// test of a null function pointer.
namespace {
struct CallRange {
    explicit CallRange(const char* name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
    CallRange(const CallRange&) = delete;
    CallRange& operator=(const CallRange&) = delete;
};
}  // namespace

extern "C" {

int32_t sdtw_abi_version(void) { return SDTW_ABI_VERSION; }

const char* sdtw_status_string(sdtw_status s)
{
    switch (s) {
    case SDTW_OK: return "SDTW_OK";
    case SDTW_E_INVALID: return "SDTW_E_INVALID: invalid argument";
    case SDTW_E_NOMEM: return "SDTW_E_NOMEM: workspace allocation failed or over the memory cap";
    case SDTW_E_CUDA: return "SDTW_E_CUDA: CUDA runtime error";
    case SDTW_E_TIMEOUT: return "SDTW_E_TIMEOUT: a bounded device wait ran out";
    case SDTW_E_UNSUPPORTED: return "SDTW_E_UNSUPPORTED: not supported by this build";
    }
    return "SDTW: unknown status";
}

sdtw_status sdtw_config_init(sdtw_config* cfg)
{
    if (!cfg) return SDTW_E_INVALID;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->dtype = SDTW_F32;
    cfg->device = 0;
    cfg->max_ref_len = 100000;
    cfg->max_total_query_len = 512 * 2000;
    cfg->max_batch = 512;
    cfg->max_query_len = 2000;
    return SDTW_OK;
}

sdtw_status sdtw_create(sdtw_ctx** out, const sdtw_config* cfg)
{
    CallRange range("sdtw_create");
    if (!out || !cfg) return SDTW_E_INVALID;
    *out = nullptr;
    if (cfg->dtype != SDTW_F32 && cfg->dtype != SDTW_I8 && cfg->dtype != SDTW_U8 && cfg->dtype != SDTW_F16)
        return SDTW_E_INVALID;
    if (cfg->max_ref_len < 1 || cfg->max_query_len < 1 || cfg->max_batch < 1 || cfg->max_total_query_len < 1)
        return SDTW_E_INVALID;
    if (cfg->max_ref_len > INT_MAX / 2) return SDTW_E_INVALID;
    if ((cfg->flags & (SDTW_FLAG_GRAD | SDTW_FLAG_KEEP_CHECKPOINTS)) && cfg->dtype != SDTW_F32) return SDTW_E_INVALID;
    if ((cfg->flags & SDTW_FLAG_KEEP_CHECKPOINTS) && !(cfg->flags & SDTW_FLAG_GRAD)) return SDTW_E_INVALID;
    if ((cfg->flags & SDTW_FLAG_ZNORM_QUERIES) && cfg->dtype != SDTW_F32) return SDTW_E_INVALID;
    if (cfg->seg_width > 0 && !sdtw::fwd_width_supported(cfg->dtype, cfg->seg_width)) return SDTW_E_INVALID;
    if (cfg->tile_rows != 0 && cfg->tile_rows != 2 && cfg->tile_rows != 4 && cfg->tile_rows != 8) return SDTW_E_INVALID;
    // 8-row tiles: 16 to 28 columns
    if (cfg->tile_rows == 8 && cfg->seg_width > 0 &&
        !sdtw::fwd_plan_supported(cfg->dtype, cfg->seg_width, 8, (cfg->flags & SDTW_FLAG_GRAD) != 0))
        return SDTW_E_INVALID;
    if (cfg->ckpt_stride < 0 || cfg->prune_gap < 0 || cfg->spin_limit != 0) return SDTW_E_INVALID;
    if (cfg->bwd_warps < 0 || cfg->bwd_warps > 4) return SDTW_E_INVALID;
    if (cfg->prune_gap > 0 && !int_mode(cfg->dtype)) return SDTW_E_INVALID;  // pruning: integer modes only
    if (cfg->ckpt_stride != 0 && !sdtw::ckpt_stride_supported(cfg->ckpt_stride)) return SDTW_E_UNSUPPORTED;
    if (cfg->warps_per_query < 0 || cfg->warps_per_query > sdtw::kMaxWarpsPerQuery) return SDTW_E_INVALID;
    if (int_mode(cfg->dtype) && cfg->max_query_len > kI8MaxN) return SDTW_E_INVALID;
    // the longest query any forward plan can stage in shared memory (one warp,
    // the smallest ring): beyond it every call would fail
    if (sdtw::fwd_smem_bytes(cfg->dtype, cfg->max_query_len, 1, 8, 4) > kMaxSmem) return SDTW_E_UNSUPPORTED;

    sdtw_ctx* c = new (std::nothrow) sdtw_ctx();
    if (!c) return SDTW_E_NOMEM;
    c->cfg = *cfg;
    c->cap = cfg->mem_cap_bytes ? cfg->mem_cap_bytes : kDefaultCap;
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, cfg->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return SDTW_E_CUDA;
    }
    sdtw_status s = dev_alloc(c, reinterpret_cast<void**>(&c->d_status), sizeof(int));
    if (s == SDTW_OK) s = dev_alloc(c, reinterpret_cast<void**>(&c->d_queue), sizeof(int));
    if (s == SDTW_OK) s = dev_alloc(c, reinterpret_cast<void**>(&c->d_order), 4 * static_cast<size_t>(cfg->max_batch));
    if (s == SDTW_OK && (cfg->flags & SDTW_FLAG_ZNORM_QUERIES))
        s = dev_alloc(c, reinterpret_cast<void**>(&c->d_zq), 4 * static_cast<size_t>(cfg->max_total_query_len));
    if (s == SDTW_OK && (cfg->flags & SDTW_FLAG_GRAD)) s = alloc_backward(c);
    if (s == SDTW_OK) {
        e = cudaMemset(c->d_status, 0, sizeof(int));
        if (e != cudaSuccess) s = cuda_fail(c, e);
    }
    if (s != SDTW_OK) {
        free_all(c);
        delete c;
        return s;
    }
    *out = c;
    return SDTW_OK;
}

sdtw_status sdtw_destroy(sdtw_ctx* ctx)
{
    if (!ctx) return SDTW_OK;
    cudaSetDevice(ctx->cfg.device);
    cudaError_t e = cudaDeviceSynchronize();
    free_all(ctx);
    delete ctx;
    return e == cudaSuccess ? SDTW_OK : SDTW_E_CUDA;
}

sdtw_status sdtw_forward(sdtw_ctx* ctx, const void* ref, int64_t M, const void* queries, const int64_t* offsets,
                         int32_t B, int32_t N, void* cost, int64_t* end, void* stream)
{
    CallRange range("sdtw_forward");
    sdtw_status s = check_common(ctx, ref, M, queries, B, N, cost, end);
    if (s != SDTW_OK) return s;
    if (offsets && ctx->cfg.dtype == SDTW_F16) return SDTW_E_UNSUPPORTED;  // binary16 pairs: uniform batches
    if (!offsets && static_cast<int64_t>(B) * N > ctx->cfg.max_total_query_len) return SDTW_E_INVALID;
    if (B == 0) return SDTW_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ctx->key.valid = false;
    const void* fq;
    if ((s = fill_queries(ctx, queries, offsets, B, N, st, &fq)) != SDTW_OK) return s;
    const FwdPlan cp = ckpt_plan(ctx, B, N, M, offsets != nullptr);
    if (keep_fits(ctx, B, N, M, cp)) {
        // store the checkpoints a following sdtw_backward on these inputs reuses
        const CkPtrs ck = carve(ctx, ck_layout(M, N, cp), B, M);
        s = run_forward(ctx, ref, M, fq, offsets, B, N, cost, end, st, &cp, &ck, 0, B);
        if (s == SDTW_OK) {
            ctx->key.ref = ref;
            ctx->key.queries = queries;
            ctx->key.offsets = offsets;
            ctx->key.M = M;
            ctx->key.B = B;
            ctx->key.N = N;
            ctx->key.W = cp.W;
            ctx->key.P = cp.P;
            ctx->key.RT = cp.RT;
            ctx->key.KS = cp.KS;
            ctx->key.valid = true;
        }
        return s;
    }
    return run_forward(ctx, ref, M, fq, offsets, B, N, cost, end, st, nullptr, nullptr, 0, B);
}

// The backward of queries q0 .. q0+nq-1 from the checkpoints in ck written by
// a forward with plan p: the band walk, then (with gradients) the reduction of
// the reference gradient.  grad_queries == nullptr: the path only.
cudaError_t launch_bwd(sdtw_ctx* ctx, const FwdPlan& p, const CkPtrs& ck, const float* ref, int64_t M,
                       const float* queries, const int64_t* offsets, int32_t B, int32_t N, const int64_t* end,
                       const float* grad_cost, float* grad_queries, float* grad_ref, int32_t* path, int q0, int nq,
                       cudaStream_t st)
{
    sdtw::BwdArgs a{};
    a.ref = ref;
    a.M = M;
    a.queries = queries;
    a.offsets = offsets;
    a.B = nq;
    a.N = N;
    a.q0 = q0;
    a.B_total = B;
    a.end = end;
    a.grad_cost = grad_cost;
    a.grad_queries = grad_queries;
    a.path = path;
    a.fr = ck.fr;
    a.fr_slot = ck.fr_slot;
    a.colck = ck.colck;
    a.ck_slot = ck.ck_slot;
    a.K = ck.K;
    a.ck_cost = ck.ck_cost;
    a.ck_end = ck.ck_end;
    a.W = p.W;
    a.P = p.P;
    a.RT = p.RT;
    a.KS = p.KS;
    a.rebase_period = sdtw::ckpt_rebase_period(p.KS);
    a.warps = ctx->cfg.bwd_warps;
    a.idle_helpers = (ctx->cfg.flags & SDTW_FLAG_TEST_IDLE_HELPERS) ? 1 : 0;
    a.gyq = ck.gyq;
    a.span = ck.span;
    a.status = ctx->d_status;
    a.q_limit = (ctx->cfg.flags & SDTW_FLAG_ZNORM_QUERIES) ? ctx->cfg.max_total_query_len : 0;
    cudaError_t e = sdtw::launch_backward_walk(a, st);
    if (e == cudaSuccess && grad_queries) e = sdtw::launch_grad_ref_reduce(ck.gyq, ck.span, nq, M, q0 > 0, grad_ref, st);
    return e;
}

// The walk-back of every query from its end column, chunk by chunk of
// queries; with grad_queries == nullptr only the path is written.
static sdtw_status run_backward(sdtw_ctx* ctx, const float* ref, int64_t M, const float* queries, const int64_t* offsets,
                         int32_t B, int32_t N, const int64_t* end, const float* grad_cost, float* grad_queries,
                         float* grad_ref, int32_t* path, cudaStream_t st)
{
    sdtw_status s;
    cudaError_t e;
    // the plan of the checkpoints: the kept forward's, or the one re-run here
    const bool reuse = key_matches(ctx->key, ref, M, queries, offsets, B, N);
    const void* fqv;
    if ((s = fill_queries(ctx, queries, offsets, B, N, st, &fqv)) != SDTW_OK) return s;
    const float* fq = static_cast<const float*>(fqv);
    FwdPlan p = ckpt_plan(ctx, B, N, M, offsets != nullptr);
    if (reuse) {
        p.W = ctx->key.W;
        p.P = ctx->key.P;
        p.RT = ctx->key.RT;
        p.KS = ctx->key.KS;
    }
    if (!sdtw::bwd_width_supported(p.W)) return SDTW_E_UNSUPPORTED;
    if (sdtw::bwd_smem_bytes(N, p.W, p.RT, p.KS) > kMaxSmem) return SDTW_E_UNSUPPORTED;
    const CkLayout l = ck_layout(M, N, p);
    const int64_t cap = chunk_capacity(ctx, l);
    if (cap < 1) return SDTW_E_NOMEM;
    const int chunk = reuse ? B : static_cast<int>(std::min<int64_t>(B, cap));
    const CkPtrs ck = carve(ctx, l, chunk, M);
    for (int q0 = 0; q0 < B; q0 += chunk) {
        const int nq = std::min(chunk, B - q0);
        if (!reuse) {
            s = run_forward(ctx, ref, M, fq, offsets, B, N, ctx->d_cost_tmp, ctx->d_end_tmp, st, &p, &ck, q0, nq);
            if (s != SDTW_OK) return s;
        }
        if ((e = launch_bwd(ctx, p, ck, ref, M, fq, offsets, B, N, end, grad_cost, grad_queries, grad_ref, path,
                            q0, nq, st)) != cudaSuccess)
            return cuda_fail(ctx, e);
    }
    // with normalised queries: the gradient with respect to the raw ones
    if (grad_queries && fq != queries &&
        (e = sdtw::launch_znorm_vjp(queries, grad_queries, offsets, B, N, ctx->cfg.max_total_query_len, st)) !=
            cudaSuccess)
        return cuda_fail(ctx, e);
    if (!reuse) ctx->key.valid = false;
    return SDTW_OK;
}

sdtw_status sdtw_backward(sdtw_ctx* ctx, const float* ref, int64_t M, const float* queries, const int64_t* offsets,
                          int32_t B, int32_t N, const int64_t* end, const float* grad_cost, float* grad_queries,
                          float* grad_ref, int32_t* path, void* stream)
{
    CallRange range("sdtw_backward");
    if (!ctx) return SDTW_E_INVALID;
    if (ctx->cfg.dtype != SDTW_F32) return SDTW_E_UNSUPPORTED;
    if (!(ctx->cfg.flags & SDTW_FLAG_GRAD)) return SDTW_E_INVALID;
    sdtw_status s = check_common(ctx, ref, M, queries, B, N, end, grad_cost);
    if (s != SDTW_OK) return s;
    if (B > 0 && (!grad_queries || !grad_ref)) return SDTW_E_INVALID;
    if (!offsets && static_cast<int64_t>(B) * N > ctx->cfg.max_total_query_len) return SDTW_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (B == 0) {
        if (!grad_ref) return SDTW_E_INVALID;
        cudaError_t e = cudaMemsetAsync(grad_ref, 0, 4 * static_cast<size_t>(M), st);
        return e == cudaSuccess ? SDTW_OK : cuda_fail(ctx, e);
    }
    return run_backward(ctx, ref, M, queries, offsets, B, N, end, grad_cost, grad_queries, grad_ref, path, st);
}

sdtw_status sdtw_path(sdtw_ctx* ctx, const float* ref, int64_t M, const float* queries, const int64_t* offsets,
                      int32_t B, int32_t N, const int64_t* end, int32_t* path, void* stream)
{
    CallRange range("sdtw_path");
    if (!ctx) return SDTW_E_INVALID;
    if (ctx->cfg.dtype != SDTW_F32) return SDTW_E_UNSUPPORTED;
    if (!(ctx->cfg.flags & SDTW_FLAG_GRAD)) return SDTW_E_INVALID;
    sdtw_status s = check_common(ctx, ref, M, queries, B, N, end, path);
    if (s != SDTW_OK) return s;
    if (!offsets && static_cast<int64_t>(B) * N > ctx->cfg.max_total_query_len) return SDTW_E_INVALID;
    if (B == 0) return SDTW_OK;
    return run_backward(ctx, ref, M, queries, offsets, B, N, end, nullptr, nullptr, nullptr, path,
                        static_cast<cudaStream_t>(stream));
}

sdtw_status sdtw_forward_host(sdtw_ctx* ctx, const void* ref, int64_t M, const void* queries, const int64_t* offsets,
                              int32_t B, int32_t N, void* cost, int64_t* end, void* stream)
{
    CallRange range("sdtw_forward_host");
    sdtw_status s = check_common(ctx, ref, M, queries, B, N, cost, end);
    if (s != SDTW_OK) return s;
    if (offsets && ctx->cfg.dtype == SDTW_F16) return SDTW_E_UNSUPPORTED;
    if (B == 0) return SDTW_OK;
    const int64_t total = offsets ? offsets[B] : static_cast<int64_t>(B) * N;
    if (total < 0 || total > ctx->cfg.max_total_query_len) return SDTW_E_INVALID;
    const size_t es = elem_size(ctx->cfg.dtype);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((s = ensure(ctx, ctx->st_ref, es * M)) != SDTW_OK) return s;
    if ((s = ensure(ctx, ctx->st_q, es * std::max<int64_t>(total, 1))) != SDTW_OK) return s;
    if ((s = ensure(ctx, ctx->st_cost, 4 * static_cast<size_t>(B))) != SDTW_OK) return s;
    if ((s = ensure(ctx, ctx->st_end, 8 * static_cast<size_t>(B))) != SDTW_OK) return s;
    if (offsets && (s = ensure(ctx, ctx->st_off, 8 * static_cast<size_t>(B + 1))) != SDTW_OK) return s;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(ctx->st_ref.p, ref, es * M, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(ctx, e);
    if (total > 0 && (e = cudaMemcpyAsync(ctx->st_q.p, queries, es * total, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(ctx, e);
    if (offsets &&
        (e = cudaMemcpyAsync(ctx->st_off.p, offsets, 8 * static_cast<size_t>(B + 1), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
        return cuda_fail(ctx, e);
    s = sdtw_forward(ctx, ctx->st_ref.p, M, ctx->st_q.p, offsets ? static_cast<const int64_t*>(ctx->st_off.p) : nullptr,
                     B, N, ctx->st_cost.p, static_cast<int64_t*>(ctx->st_end.p), stream);
    if (s != SDTW_OK) return s;
    if ((e = cudaMemcpyAsync(cost, ctx->st_cost.p, 4 * static_cast<size_t>(B), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(ctx, e);
    if ((e = cudaMemcpyAsync(end, ctx->st_end.p, 8 * static_cast<size_t>(B), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(ctx, e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(ctx, e);
    ctx->key.valid = false;  // staged inputs are reused by later host calls
    return SDTW_OK;
}

sdtw_status sdtw_forward_backward_host(sdtw_ctx* ctx, const float* ref, int64_t M, const float* queries,
                                       const int64_t* offsets, int32_t B, int32_t N, const float* grad_cost,
                                       float* cost, int64_t* end, float* grad_queries, float* grad_ref,
                                       int32_t* path, void* stream)
{
    CallRange range("sdtw_forward_backward_host");
    if (!ctx) return SDTW_E_INVALID;
    if (ctx->cfg.dtype != SDTW_F32) return SDTW_E_UNSUPPORTED;
    if (!(ctx->cfg.flags & SDTW_FLAG_GRAD)) return SDTW_E_INVALID;
    sdtw_status s = check_common(ctx, ref, M, queries, B, N, cost, end);
    if (s != SDTW_OK) return s;
    if (B > 0 && (!grad_cost || !grad_queries)) return SDTW_E_INVALID;
    if (!grad_ref) return SDTW_E_INVALID;
    const int64_t total = B == 0 ? 0 : (offsets ? offsets[B] : static_cast<int64_t>(B) * N);
    if (total < 0 || total > ctx->cfg.max_total_query_len) return SDTW_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if ((s = ensure(ctx, ctx->st_ref, 4 * M)) != SDTW_OK) return s;
    if ((s = ensure(ctx, ctx->st_q, 4 * std::max<int64_t>(total, 1))) != SDTW_OK) return s;
    if ((s = ensure(ctx, ctx->st_cost, 4 * static_cast<size_t>(std::max(B, 1)))) != SDTW_OK) return s;
    if ((s = ensure(ctx, ctx->st_end, 8 * static_cast<size_t>(std::max(B, 1)))) != SDTW_OK) return s;
    if ((s = ensure(ctx, ctx->st_gc, 4 * static_cast<size_t>(std::max(B, 1)))) != SDTW_OK) return s;
    if ((s = ensure(ctx, ctx->st_gq, 4 * std::max<int64_t>(total, 1))) != SDTW_OK) return s;
    if ((s = ensure(ctx, ctx->st_gr, 4 * M)) != SDTW_OK) return s;
    if (path && (s = ensure(ctx, ctx->st_path, 8 * std::max<int64_t>(total, 1))) != SDTW_OK) return s;
    if (offsets && (s = ensure(ctx, ctx->st_off, 8 * static_cast<size_t>(B + 1))) != SDTW_OK) return s;
    if ((e = cudaMemcpyAsync(ctx->st_ref.p, ref, 4 * M, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(ctx, e);
    if (total > 0 && (e = cudaMemcpyAsync(ctx->st_q.p, queries, 4 * total, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(ctx, e);
    if (B > 0 && (e = cudaMemcpyAsync(ctx->st_gc.p, grad_cost, 4 * static_cast<size_t>(B), cudaMemcpyHostToDevice, st)) !=
                     cudaSuccess)
        return cuda_fail(ctx, e);
    if (offsets &&
        (e = cudaMemcpyAsync(ctx->st_off.p, offsets, 8 * static_cast<size_t>(B + 1), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
        return cuda_fail(ctx, e);
    const int64_t* doff = offsets ? static_cast<const int64_t*>(ctx->st_off.p) : nullptr;
    const float* dref = static_cast<const float*>(ctx->st_ref.p);
    const float* dq = static_cast<const float*>(ctx->st_q.p);
    s = sdtw_forward(ctx, dref, M, dq, doff, B, N, ctx->st_cost.p, static_cast<int64_t*>(ctx->st_end.p), stream);
    if (s != SDTW_OK) return s;
    s = sdtw_backward(ctx, dref, M, dq, doff, B, N, static_cast<const int64_t*>(ctx->st_end.p),
                      static_cast<const float*>(ctx->st_gc.p), static_cast<float*>(ctx->st_gq.p),
                      static_cast<float*>(ctx->st_gr.p), path ? static_cast<int32_t*>(ctx->st_path.p) : nullptr, stream);
    if (s != SDTW_OK) return s;
    if (B > 0) {
        if ((e = cudaMemcpyAsync(cost, ctx->st_cost.p, 4 * static_cast<size_t>(B), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(ctx, e);
        if ((e = cudaMemcpyAsync(end, ctx->st_end.p, 8 * static_cast<size_t>(B), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(ctx, e);
        if ((e = cudaMemcpyAsync(grad_queries, ctx->st_gq.p, 4 * total, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(ctx, e);
        if (path && (e = cudaMemcpyAsync(path, ctx->st_path.p, 8 * total, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(ctx, e);
    }
    if ((e = cudaMemcpyAsync(grad_ref, ctx->st_gr.p, 4 * M, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(ctx, e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(ctx, e);
    ctx->key.valid = false;
    return SDTW_OK;
}

sdtw_status sdtw_autotune(sdtw_ctx* ctx, const void* ref, int64_t M, const void* queries, const int64_t* offsets,
                          int32_t B, int32_t N, void* cost, int64_t* end, void* stream, sdtw_plan* plan)
{
    CallRange range("sdtw_autotune");
    sdtw_status s = check_common(ctx, ref, M, queries, B, N, cost, end);
    if (s != SDTW_OK) return s;
    if (offsets && ctx->cfg.dtype == SDTW_F16) return SDTW_E_UNSUPPORTED;
    if (B == 0) return SDTW_E_INVALID;
    if (!offsets && static_cast<int64_t>(B) * N > ctx->cfg.max_total_query_len) return SDTW_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool ragged = offsets != nullptr;
    // every timed run reads the queries the fill would read
    if ((s = fill_queries(ctx, queries, offsets, B, N, st, &queries)) != SDTW_OK) return s;
    // with kept checkpoints, time the checkpointing forward (its stores
    // included) and the backward that follows it, among the plans whose
    // checkpoints fit the arena: the plan then serves the differentiable step
    const bool ckpt = keep_fits(ctx, B, N, M, ckpt_plan(ctx, B, N, M, ragged));
    float *t_gc = nullptr, *t_gq = nullptr, *t_gr = nullptr;  // gradient scratch of the timed backward
    auto free_scratch = [&]() {
        cudaFree(t_gc);
        cudaFree(t_gq);
        cudaFree(t_gr);
    };
    if (ckpt && ctx->cfg.dtype == SDTW_F32) {
        const size_t nqs = offsets ? static_cast<size_t>(ctx->cfg.max_total_query_len) : static_cast<size_t>(B) * N;
        if (cudaMalloc(&t_gc, 4 * static_cast<size_t>(B)) != cudaSuccess ||
            cudaMalloc(&t_gq, 4 * std::max<size_t>(nqs, 1)) != cudaSuccess ||
            cudaMalloc(&t_gr, 4 * static_cast<size_t>(M)) != cudaSuccess ||
            cudaMemsetAsync(t_gc, 0, 4 * static_cast<size_t>(B), st) != cudaSuccess) {
            cudaGetLastError();
            free_scratch();
            return SDTW_E_NOMEM;
        }
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        free_scratch();
        return SDTW_E_CUDA;
    }
    float best_ms = 1e30f;
    int best_w = 0, best_p = 0, best_rt = 0, best_ks = 0;
    const int Ws[] = {8, 16, 20, 24, 28, 32};
    const int Ps[] = {1, 2, 3, 4, 5, 6, 7, 8, 16};
    const int RTs[] = {2, 4, 8};
    // the checkpoint stride is an axis only when checkpoints are stored (and
    // the caller did not fix it); a stride whose checkpoints do not fit the
    // arena under the memory cap is skipped like any other plan
    std::vector<int> KSs;
    if (!ckpt) KSs.push_back(kDefaultStride);
    else if (ctx->cfg.ckpt_stride > 0) KSs.push_back(ctx->cfg.ckpt_stride);
    else KSs.assign(std::begin(kStrides), std::end(kStrides));
    for (int KS : KSs) {
    for (int RT : RTs) {
        for (int W : Ws) {
            for (int P : Ps) {
                if (static_cast<int64_t>(32) * P * W > 4 * M && P > 1) continue;
                if (!sdtw::fwd_plan_supported(ctx->cfg.dtype, W, RT, ckpt)) continue;
                FwdPlan p = default_fwd_plan(ctx, B, N, M, ragged, ckpt);
                p.W = W;
                p.P = P;
                p.RT = RT;
                p.KS = KS;
                p.block = 32 * P;
                p.smem = sdtw::fwd_smem_bytes(ctx->cfg.dtype, N, P, W, RT);
                if (p.smem > kMaxSmem) continue;
                const CkLayout l = ck_layout(M, N, p);
                if (ckpt && B > chunk_capacity(ctx, l)) continue;
                const CkPtrs ck = ckpt ? carve(ctx, l, B, M) : CkPtrs{};
                const bool with_bwd = t_gc && sdtw::bwd_width_supported(W) &&
                                      sdtw::bwd_smem_bytes(N, W, RT, KS) <= kMaxSmem;
                if (t_gc && !with_bwd) continue;  // a plan the backward cannot use
                const int per_sm = sdtw::fwd_max_ctas_per_sm(ctx->cfg.dtype, W, P, p.smem, RT, ckpt, ctx->cfg.prune_gap > 0);
                if (per_sm <= 0) continue;
                p.grid = p.persistent ? std::max(1, std::min(B, per_sm * ctx->sm_count)) : plain_grid(ctx->cfg.dtype, B);
                // one untimed run, then the best of two timed runs
                float ms = 1e30f;
                for (int rep = 0; rep < 3; ++rep) {
                    cudaEventRecord(e0, st);
                    s = run_forward(ctx, ref, M, queries, offsets, B, N, cost, end, st, &p, ckpt ? &ck : nullptr,
                                    0, B);
                    if (s == SDTW_OK && with_bwd &&
                        launch_bwd(ctx, p, ck, static_cast<const float*>(ref), M, static_cast<const float*>(queries),
                                   offsets, B, N, end, t_gc, t_gq, t_gr, nullptr, 0, B, st) != cudaSuccess)
                        s = SDTW_E_CUDA;
                    cudaEventRecord(e1, st);
                    if (s != SDTW_OK) break;
                    if (cudaEventSynchronize(e1) != cudaSuccess) {
                        s = SDTW_E_CUDA;
                        break;
                    }
                    float t = 0;
                    cudaEventElapsedTime(&t, e0, e1);
                    if (rep > 0) ms = std::min(ms, t);
                }
                if (s == SDTW_E_UNSUPPORTED) {
                    s = SDTW_OK;
                    continue;
                }
                if (s != SDTW_OK) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    free_scratch();
                    return s;
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best_w = W;
                    best_p = P;
                    best_rt = RT;
                    best_ks = KS;
                }
            }
        }
    }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    free_scratch();
    if (best_w == 0) return SDTW_E_UNSUPPORTED;
    ctx->tuned[TuneKey{ctx->cfg.dtype, ragged ? 1 : 0, bucket_of(N), bucket_of(M), ckpt ? 1 : 0}] =
        std::make_tuple(best_w, best_p, best_rt, best_ks);
    ctx->key.valid = false;
    if (plan) return sdtw_get_plan(ctx, B, N, M, ragged ? 1 : 0, 0, plan);
    return SDTW_OK;
}

sdtw_status sdtw_get_plan(sdtw_ctx* ctx, int32_t B, int32_t N, int64_t M, int32_t ragged, int32_t backward,
                          sdtw_plan* plan)
{
    if (!ctx || !plan || B < 1 || N < 1 || M < 1) return SDTW_E_INVALID;
    if (backward && !(ctx->cfg.flags & SDTW_FLAG_GRAD)) return SDTW_E_INVALID;
    const bool ckpt = backward || keep_fits(ctx, B, N, M, ckpt_plan(ctx, B, N, M, ragged != 0));
    FwdPlan p = default_fwd_plan(ctx, B, N, M, ragged != 0, ckpt);
    std::memset(plan, 0, sizeof(*plan));
    plan->seg_width = p.W;
    plan->warps_per_query = p.P;
    plan->ctas_per_query = 1;
    plan->persistent = p.persistent ? 1 : 0;
    plan->grid = p.persistent ? p.grid : plain_grid(ctx->cfg.dtype, B);
    plan->block = p.block;
    plan->smem_bytes = static_cast<int32_t>(std::min<int64_t>(p.smem, INT32_MAX));
    plan->ckpt_stride = ckpt ? p.KS : 0;
    plan->ckpt_cols = ckpt ? 8 * p.W : 0;
    plan->tuned = ctx->tuned.count(TuneKey{ctx->cfg.dtype, ragged ? 1 : 0, bucket_of(N), bucket_of(M), ckpt ? 1 : 0})
                      ? 1
                      : 0;
    plan->sweep_cols = static_cast<int64_t>(32) * p.P * p.W;
    plan->tile_rows = p.RT;
    plan->bwd_warps = backward ? sdtw::bwd_warps(N, p.W, p.RT, p.KS, ctx->cfg.bwd_warps) : 0;
    return SDTW_OK;
}

sdtw_status sdtw_last_device_status(sdtw_ctx* ctx, void* stream)
{
    if (!ctx) return SDTW_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    int v = 0;
    if ((e = cudaMemcpy(&v, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(ctx, e);
    if (v != 0 && (e = cudaMemset(ctx->d_status, 0, sizeof(int))) != cudaSuccess) return cuda_fail(ctx, e);
    if (v & sdtw::kStatusTimeout) return SDTW_E_TIMEOUT;
    if (v) return SDTW_E_INVALID;
    return SDTW_OK;
}

const char* sdtw_last_error(sdtw_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

size_t sdtw_workspace_bytes(sdtw_ctx* ctx) { return ctx ? ctx->ws_bytes : 0; }

}  // extern "C"
