// qt_api.cu -- host side of libqt: contexts, workspace, descriptor tables,
// CUDA-graph capture of the forward step, the autotuner, and every C-ABI entry
// point declared in include/qt.h.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/qt.h"
#include "qt_internal.h"
#include "qt_launch.h"

namespace qt {
__global__ void prep_records_kernel(const double*, GridInfo*, int, int, int, int, long long, float*, double*);
__global__ void backward_layer_kernel(const void*, int, long long, int, int, const double*, const double*, double*);
__global__ void root_price_kernel(const void*, int, int, int, const double*, double*);
__global__ void fold_status_kernel(const DevStatus*, DevStatus*);
__global__ void swing_terminal_kernel(int, int, int, int, double*);
__global__ void swing_layer_kernel(const void*, int, long long, int, int, const double*, const double*, double*, int,
                                   int, int, int);
__global__ void kmeans_draw_kernel(int, unsigned long long, long long, float*);
__global__ void kmeans_assign_kernel(int, long long, const float*, int, const float*, unsigned long long*,
                                     unsigned long long*, int);
__global__ void kmeans_update_kernel(int, int, const unsigned long long*, const unsigned long long*, float*);
__global__ void map_grid_kernel(int, int, const double*, const double*, const double*, double*);
__global__ void prep_tc_tiles_kernel(const float*, GridInfo*, int, int, int, int, int, long long, __half*);
cudaError_t launch_router_forward(int dm, const ForwardParams& p, int num_sms, int* bps, cudaStream_t st);
cudaError_t launch_grid_checksum(const double* grids, long long count, unsigned long long* out, cudaStream_t st);
void router_fill_params(const qt_router* r, ForwardParams& fp);
bool router_matches(const qt_router* r, int d, int n, const int64_t* N);
}  // namespace qt

using namespace qt;

// ------------------------------------------------------------------ context

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct HostBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct TuneKey {
    int form, dm, prec, nbucket;
    bool operator<(const TuneKey& o) const
    {
        return std::tie(form, dm, prec, nbucket) < std::tie(o.form, o.dm, o.prec, o.nbucket);
    }
};

}  // namespace

struct qt_ctx {
    int device = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    std::string err;
    std::map<std::string, DevBuf> dev;
    std::map<std::string, HostBuf> host;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t ev_tables = nullptr;   // last use of the pinned descriptor tables
    cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;   // around the forward kernel (stats.ms)
    bool timed = false;
    // cached graph of the last forward call
    cudaGraphExec_t gexec = nullptr;
    std::vector<unsigned char> gkey;
    // autotuner cache: key -> samples per thread
    std::map<TuneKey, int> tune;
    int last_form = 0;
    int last_launches = 0;             // kernels enqueued by the last forward step
    int last_tc_draw = 0;              // sample-draw layout of the last tensor-core step
    void* status_buf = nullptr;   // status block of the last forward call
};

namespace {

qt_status fail(qt_ctx* c, qt_status s, const char* fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define QT_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? QT_ENOMEM : QT_ECUDA, "%s: %s", \
                        #call, cudaGetErrorString(e_));                                        \
        }                                                                                      \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int now = -1;
        cudaGetDevice(&now);
        if (prev >= 0 && now != prev) cudaSetDevice(prev);
    }
};

// Host-side fault injection for the allocation-failure tests: QT_FAULT=alloc
// makes the next workspace allocation fail as if the device were out of memory.
bool injected_alloc_failure()
{
    const char* f = getenv("QT_FAULT");
    return f && strcmp(f, "alloc") == 0;
}

// QT_FAULT=timeout_layer:K gives the launch that runs layer pair K alone (the
// fused price mode) a negative wait budget, so that its first bounded wait
// gives up as if the copy never landed: a timeout in one layer only.
int injected_timeout_layer()
{
    const char* f = getenv("QT_FAULT");
    if (!f || strncmp(f, "timeout_layer:", 14) != 0) return -1;
    return atoi(f + 14);
}

qt_status dev_get(qt_ctx* ctx, const char* name, size_t bytes, void** out)
{
    DevBuf& b = ctx->dev[name];
    if (b.bytes < bytes) {
        if (injected_alloc_failure()) return fail(ctx, QT_ENOMEM, "workspace '%s': injected allocation failure", name);
        if (b.p) cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
        size_t want = std::max<size_t>(bytes, 256);
        cudaError_t e = cudaMalloc(&b.p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            return fail(ctx, QT_ENOMEM, "workspace '%s' (%zu bytes): %s", name, want, cudaGetErrorString(e));
        }
        b.bytes = want;
        // a workspace that moved invalidates the cached graph
        if (ctx->gexec) {
            cudaGraphExecDestroy(ctx->gexec);
            ctx->gexec = nullptr;
            ctx->gkey.clear();
        }
    }
    *out = b.p;
    return QT_OK;
}

qt_status host_get(qt_ctx* ctx, const char* name, size_t bytes, void** out)
{
    HostBuf& b = ctx->host[name];
    if (b.bytes < bytes) {
        if (ctx->ev_tables) cudaEventSynchronize(ctx->ev_tables);
        if (b.p) cudaFreeHost(b.p);
        b.p = nullptr;
        b.bytes = 0;
        size_t want = std::max<size_t>(bytes, 256);
        cudaError_t e = cudaMallocHost(&b.p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, QT_ENOMEM, "pinned host buffer '%s': %s", name, cudaGetErrorString(e));
        }
        b.bytes = want;
        if (ctx->gexec) {
            cudaGraphExecDestroy(ctx->gexec);
            ctx->gexec = nullptr;
            ctx->gkey.clear();
        }
    }
    *out = b.p;
    return QT_OK;
}

qt_status validate_model(qt_ctx* ctx, const qt_model* m)
{
    if (!m) return fail(ctx, QT_EINVAL, "model is NULL");
    if (m->d < 1 || m->d > kDMax) return fail(ctx, QT_EINVAL, "d = %d outside [1, %d]", m->d, kDMax);
    if (m->n < 1 || m->n > 65535) return fail(ctx, QT_EINVAL, "n = %d outside [1, 65535]", m->n);
    if (!m->N || !m->A || !m->b || !m->T || !m->m || !m->L) return fail(ctx, QT_EINVAL, "model array is NULL");
    for (int k = 0; k <= m->n; ++k)
        if (m->N[k] < 1 || m->N[k] > (1 << 24)) return fail(ctx, QT_EINVAL, "N[%d] = %lld outside [1, 2^24]", k, (long long)m->N[k]);
    return QT_OK;
}

int dm_for(int d)
{
    static const int dms[] = {1, 2, 3, 4, 6, 8, 10, 12, 16};
    for (int v : dms)
        if (v >= d) return v;
    return 0;
}

int rec_floats_for(int dm) { return 4 * ((dm + 1 + 3) / 4); }
int rec64_for(int dm) { return (dm + 1) / 2 * 2; }
long long round_up(long long a, long long b) { return (a + b - 1) / b * b; }

}  // namespace

// ------------------------------------------------------------------ public: context

extern "C" qt_status qt_create(qt_ctx** out, int32_t device)
{
    qt_ctx* ctx = nullptr;
    if (!out) return QT_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return QT_ECUDA;
    }
    if (device < 0 || device >= ndev) return QT_EINVAL;
    ctx = new (std::nothrow) qt_ctx();
    if (!ctx) return QT_ENOMEM;
    ctx->device = device;
    DeviceGuard g(device);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete ctx;
        return QT_ECUDA;
    }
    if (prop.major * 10 + prop.minor < 100) {
        delete ctx;
        return QT_EUNSUPPORTED;
    }
    ctx->num_sms = prop.multiProcessorCount;
    ctx->smem_optin = prop.sharedMemPerBlockOptin;
    if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_tables, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&ctx->ev_k0) != cudaSuccess || cudaEventCreate(&ctx->ev_k1) != cudaSuccess) {
        delete ctx;
        return QT_ECUDA;
    }
    *out = ctx;
    return QT_OK;
}

extern "C" qt_status qt_destroy(qt_ctx* ctx)
{
    if (!ctx) return QT_OK;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    for (auto& kv : ctx->dev)
        if (kv.second.p) cudaFree(kv.second.p);
    for (auto& kv : ctx->host)
        if (kv.second.p) cudaFreeHost(kv.second.p);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->ev_tables) cudaEventDestroy(ctx->ev_tables);
    if (ctx->ev_k0) cudaEventDestroy(ctx->ev_k0);
    if (ctx->ev_k1) cudaEventDestroy(ctx->ev_k1);
    delete ctx;
    return QT_OK;
}

extern "C" const char* qt_last_error(const qt_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

extern "C" const char* qt_status_string(qt_status s)
{
    switch (s) {
    case QT_OK: return "ok";
    case QT_EINVAL: return "invalid argument";
    case QT_ENOMEM: return "out of memory";
    case QT_ECUDA: return "CUDA error";
    case QT_ETIMEOUT: return "device wait timed out";
    case QT_EUNSUPPORTED: return "unsupported";
    case QT_EDEVICE: return "device-side error";
    default: return "unknown status";
    }
}

extern "C" void qt_default_options(qt_options* o)
{
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->form = QT_FORM_AUTO;
    o->sample_prec = QT_PREC_F32;
    o->counts_type = QT_COUNTS_I64;
}

// ------------------------------------------------------------------ forward step

namespace {

struct Plan {
    int form = 0, dm = 0, S = 0, block = 256;
    bool streamed = false;
    int seg_records = 0;
    int tc_k = 0, tc_slots = 0, tc_resident = 0;
    long long tc_total_tiles = 0;
    long long tc_chunk_items = 0;      // tensor-core form: work items per launch
    int tc_draw_in = 0;                // tensor-core form: 1 = the screen kernel draws its samples
    size_t tc_item_bytes = 0;          // tensor-core form: drawn-sample bytes per work item
    int d = 0, n = 0, ngrids = 0;
    int euler = 0;                     // path-wise form: Euler-scheme chain
    long long total_recs = 0;
    size_t grid_bytes = 0, hist_bytes = 0, dyn_smem = 0;
    long long total_items = 0;
    int tile = 0;
    int rec_floats = 0, rec64 = 0, pstride = 0;
    std::vector<LayerDesc> layers;
    std::vector<GridInfo> grids;
    long long count_entries = 0;
};

struct FwdIO {
    const double* g64;           // concatenated FP64 grids (caller's or workspace copy)
    const float* params_f_host;  // not used directly
    void* counts;
    const qt_dump* dump;
    const double* srcX;
    const double* srcY;
    int32_t* cellsA;
    int32_t* cellsB;
};

qt_status make_plan_full(qt_ctx* ctx, int d, int n, const int64_t* Ns, const double* mus, long long M,
                         const qt_options* o, bool from_arrays, Plan& P, int algo);

// Work items per launch of the tensor-core form: all of them when the screen
// kernel draws its own samples, as many as 2 GiB of drawn samples hold with the
// draw pass, or fewer when the caller caps it.
long long tc_chunk(const Plan& P, const qt_options* o)
{
    long long c = P.total_items;
    if (!P.tc_draw_in) c = std::min<long long>(c, (2ll << 30) / (long long)P.tc_item_bytes);
    if (o->tc_chunk_items > 0) c = std::min<long long>(c, o->tc_chunk_items);
    return std::max<long long>(1, c);
}

// The plan of the whole model, or of layer pair `only_layer` alone: the other
// layers keep their descriptors (so that every kernel still finds layer k by
// its global index, which also keys the sampler's counters) but get no work
// items, and layer k's counts start at offset 0 of the counts buffer.
qt_status make_plan(qt_ctx* ctx, int d, int n, const int64_t* Ns, const double* mus, long long M, const qt_options* o,
                    bool from_arrays, Plan& P, int only_layer = -1, int algo = 3)
{
    qt_status s = make_plan_full(ctx, d, n, Ns, mus, M, o, from_arrays, P, algo);
    if (!s && algo == 2 && only_layer >= 0) return fail(ctx, QT_EUNSUPPORTED, "the path-wise form runs every layer");
    if (s || only_layer < 0) return s;
    if (only_layer >= n) return fail(ctx, QT_EINVAL, "layer %d of %d", only_layer, n);
    const int items = P.layers[only_layer].items;
    for (int k = 0; k < n; ++k) {
        P.layers[k].item_begin = k <= only_layer ? 0 : items;
        if (k != only_layer) P.layers[k].items = 0;
    }
    P.layers[only_layer].coff = 0;
    P.total_items = items;
    P.count_entries = (long long)P.layers[only_layer].NA * P.layers[only_layer].NB;
    if (P.form == kTcRecheck) P.tc_chunk_items = tc_chunk(P, o);
    return QT_OK;
}

// Pick form, dimension class, tile and shared memory for a problem described
// by grid sizes Ns (n+1 entries) and centres mus ((n+1) x d).  algo = 3 is
// Algorithm III (independent layer pairs), algo = 2 Algorithm II (paths).
qt_status make_plan_full(qt_ctx* ctx, int d, int n, const int64_t* Ns, const double* mus, long long M,
                         const qt_options* o, bool from_arrays, Plan& P, int algo)
{
    P.d = d;
    P.n = n;
    P.dm = dm_for(d);
    int form = o->form;
    if (algo == 2) {
        // the path-wise form screens in FP32 with the exact recheck
        if (form != QT_FORM_AUTO && form != QT_FORM_F32_RECHECK)
            return fail(ctx, QT_EUNSUPPORTED, "the path-wise form supports the FP32 screen only (form %d)", form);
        if (from_arrays) return fail(ctx, QT_EUNSUPPORTED, "the path-wise form draws its own paths");
        form = QT_FORM_F32_RECHECK;
    }
    // automatic choice: the fastest certified form measured on GB300 -- the
    // tensor-core screen for 3 <= d <= 10, the FP32 screen otherwise
    if (form == QT_FORM_AUTO) form = (d >= 3 && d <= 10) ? QT_FORM_TC_RECHECK : QT_FORM_F32_RECHECK;
    if (form != QT_FORM_PLAIN_F64 && form != QT_FORM_F32_RECHECK && form != QT_FORM_TC_RECHECK &&
        form != QT_FORM_ROUTER_CERT)
        return fail(ctx, QT_EINVAL, "unknown search form %d", form);
    P.form = form == QT_FORM_PLAIN_F64 ? kPlainF64
                                       : (form == QT_FORM_TC_RECHECK ? kTcRecheck
                                                                     : (form == QT_FORM_ROUTER_CERT ? kRouterCert
                                                                                                    : kF32Recheck));
    if (P.form == kRouterCert) {
        const qt_router* rt = static_cast<const qt_router*>(o->router);
        if (!rt) return fail(ctx, QT_EINVAL, "QT_FORM_ROUTER_CERT needs opts->router");
        if (from_arrays) return fail(ctx, QT_EUNSUPPORTED, "the router form draws its own samples");
        if (o->sample_prec != QT_PREC_F32) return fail(ctx, QT_EUNSUPPORTED, "the router form uses FP32 samples");
        if (!router_matches(rt, d, n, Ns)) return fail(ctx, QT_EINVAL, "model shape differs from the router's");
        P.dm = d <= 2 ? 2 : (d <= 4 ? 4 : (d <= 6 ? 6 : (d <= 8 ? 8 : (d <= 10 ? 10 : (d <= 12 ? 12 : 16)))));
    }
    if (P.form == kTcRecheck) {
        if (d > 10) return fail(ctx, QT_EUNSUPPORTED, "the tensor-core screen needs d <= 10 (3d + 2 <= 32 columns)");
        P.dm = d <= 2 ? 2 : (d <= 4 ? 4 : (d <= 6 ? 6 : (d <= 8 ? 8 : 10)));
    }
    if (!from_arrays && o->sample_prec != QT_PREC_F32 && o->sample_prec != QT_PREC_F64)
        return fail(ctx, QT_EINVAL, "sample_prec %d", o->sample_prec);
    P.rec_floats = rec_floats_for(P.dm);
    P.rec64 = rec64_for(P.dm);
    P.pstride = param_stride(d);
    P.ngrids = n + 1;
    P.grids.resize(P.ngrids);
    long long goff = 0, roff = 0;
    for (int g = 0; g < P.ngrids; ++g) {
        GridInfo& G = P.grids[g];
        memset(&G, 0, sizeof G);
        for (int l = 0; l < d; ++l) G.mu[l] = (float)mus[(long long)g * d + l];
        G.R = 0.0f;
        G.N = (int)Ns[g];
        G.Npad = P.form != kPlainF64 ? (int)round_up(Ns[g], kChunk) : (int)Ns[g];
        G.goff = goff;
        G.roff = roff;
        G.tc_tiles = (int)((Ns[g] + kTcTileN - 1) / kTcTileN);
        G.tc_toff = P.tc_total_tiles;
        if (P.form == kTcRecheck) P.tc_total_tiles += G.tc_tiles;
        goff += Ns[g];
        roff += G.Npad;
    }
    P.total_recs = roff;
    if (algo == 2) {
        // Algorithm II: a CTA carries a tile of paths through every layer; the
        // FP32 records of one grid per shared-memory buffer, two buffers
        const bool f32 = o->sample_prec == QT_PREC_F32;
        P.form = kPathwise;
        const size_t rec_bytes = (size_t)P.rec_floats * 4;
        long long npmax = 0;
        for (int g = 0; g <= n; ++g) npmax = std::max<long long>(npmax, P.grids[g].Npad);
        const size_t budget = ctx->smem_optin > 24 * 1024 ? ctx->smem_optin - 24 * 1024 : 0;
        // segments of whole grids when the largest fits half the shared memory,
        // else the largest multiple of a chunk that does
        long long seg = npmax;
        if (2 * round_up(seg * (long long)rec_bytes, 128) > (long long)budget)
            seg = (long long)(budget / 2 / rec_bytes) / kChunk * kChunk;
        if (seg < kChunk) return fail(ctx, QT_EUNSUPPORTED, "records too large for the path-wise segments");
        P.seg_records = (int)seg;
        P.streamed = seg < npmax;
        P.grid_bytes = 2 * round_up(seg * (long long)rec_bytes, 128);
        int S = o->tile_samples_per_thread > 0 ? o->tile_samples_per_thread
                                                : pathwise_default_spt(P.dm, f32, P.streamed, M, 2ll * ctx->num_sms);
        if (!pathwise_variant_exists(P.dm, S, f32, P.streamed))
            return fail(ctx, QT_EUNSUPPORTED, "no path-wise kernel for d %d, %d paths per thread", d, S);
        P.S = S;
        P.block = 256;
        P.tile = P.block * S;
        P.hist_bytes = 0;
        P.dyn_smem = P.grid_bytes;
        P.layers.resize(n);
        long long coff = 0;
        for (int k = 0; k < n; ++k) {
            LayerDesc& L = P.layers[k];
            memset(&L, 0, sizeof L);
            L.NA = (int)Ns[k];
            L.NB = (int)Ns[k + 1];
            L.NApad = P.grids[k].Npad;
            L.NBpad = P.grids[k + 1].Npad;
            L.gridA = k;
            L.gridB = k + 1;
            L.goffA = P.grids[k].goff;
            L.goffB = P.grids[k + 1].goff;
            L.roffA = P.grids[k].roff;
            L.roffB = P.grids[k + 1].roff;
            L.coff = coff;
            coff += (long long)L.NA * L.NB;
        }
        P.total_items = (M + P.tile - 1) / P.tile;
        P.count_entries = coff;
        return QT_OK;
    }
    if (P.form == kRouterCert) {
        P.S = 1;
        P.block = 128;
        P.tile = 128;
        P.grid_bytes = 0;
        P.hist_bytes = 0;
        P.dyn_smem = 0;
        P.layers.resize(n);
        long long item = 0, coff = 0;
        const long long items_per_layer = (M + P.tile - 1) / P.tile;
        for (int k = 0; k < n; ++k) {
            LayerDesc& L = P.layers[k];
            memset(&L, 0, sizeof L);
            L.NA = (int)Ns[k];
            L.NB = (int)Ns[k + 1];
            L.NApad = P.grids[k].Npad;
            L.NBpad = P.grids[k + 1].Npad;
            L.gridA = k;
            L.gridB = k + 1;
            L.goffA = P.grids[k].goff;
            L.goffB = P.grids[k + 1].goff;
            L.roffA = P.grids[k].roff;
            L.roffB = P.grids[k + 1].roff;
            L.coff = coff;
            L.item_begin = item;
            L.items = (int)items_per_layer;
            item += items_per_layer;
            coff += (long long)L.NA * L.NB;
        }
        P.total_items = item;
        P.count_entries = coff;
        return QT_OK;
    }
    if (P.form == kTcRecheck) {
        // one CTA of 16 warps per SM owns the 512 TMEM columns (four 128-column
        // accumulators); the operand tiles take what the pipeline's buffers
        // leave of the shared memory, at most 16 tiles
        P.tc_k = P.dm <= 4 ? 16 : 32;
        const size_t tile_bytes = (size_t)kTcTileN * P.tc_k * 2;
        const long long fixed = tc_fixed_smem(P.dm, P.tc_k);
        const long long room = (long long)ctx->smem_optin - fixed - 2048;
        P.tc_slots = (int)std::min<long long>(kTcMaxSlots, room > 0 ? room / (long long)tile_bytes : 0);
        if (P.tc_slots < 2) return fail(ctx, QT_EUNSUPPORTED, "too little shared memory for the tensor-core form");
        int tmax = 0;
        for (int k = 0; k < n; ++k) tmax = std::max(tmax, P.grids[k].tc_tiles + P.grids[k + 1].tc_tiles);
        P.tc_resident = tmax <= P.tc_slots;
        // resident tiles take only the slots they need: the rest of the unified
        // L1/shared memory caches the FP32 records that the certifiers re-score
        if (P.tc_resident) P.tc_slots = std::max(2, tmax);
        P.S = 1;
        P.block = kTcThreads;
        P.tile = kTcTileM;
        // where the samples are drawn: the caller's choice, else the autotuned
        // one (the caller passes it through tc_draw), else in the screen kernel
        P.tc_draw_in = o->tc_draw != 1;
        P.tc_item_bytes = (size_t)(tc_item_op_bytes(P.tc_k) + tc_item_cert_bytes(P.dm));
        P.grid_bytes = (size_t)fixed + (size_t)P.tc_slots * tile_bytes;
        P.hist_bytes = 0;
        P.dyn_smem = P.grid_bytes;
        P.layers.resize(n);
        long long item = 0, coff = 0;
        const long long items_per_layer = (M + P.tile - 1) / P.tile;
        for (int k = 0; k < n; ++k) {
            LayerDesc& L = P.layers[k];
            memset(&L, 0, sizeof L);
            L.NA = (int)Ns[k];
            L.NB = (int)Ns[k + 1];
            L.NApad = P.grids[k].Npad;
            L.NBpad = P.grids[k + 1].Npad;
            L.gridA = k;
            L.gridB = k + 1;
            L.goffA = P.grids[k].goff;
            L.goffB = P.grids[k + 1].goff;
            L.roffA = P.grids[k].roff;
            L.roffB = P.grids[k + 1].roff;
            L.coff = coff;
            L.item_begin = item;
            L.items = (int)items_per_layer;
            item += items_per_layer;
            coff += (long long)L.NA * L.NB;
        }
        P.total_items = item;
        P.tc_chunk_items = tc_chunk(P, o);
        P.count_entries = coff;
        return QT_OK;
    }
    const size_t rec_bytes = P.form == kF32Recheck ? (size_t)P.rec_floats * 4 : (size_t)P.rec64 * 8;
    // shared memory: both grids resident when they fit, else the streamed ring
    size_t budget = ctx->smem_optin > 24 * 1024 ? ctx->smem_optin - 24 * 1024 : 0;
    size_t gmax = 0;
    for (int k = 0; k < n; ++k) {
        const size_t b = (size_t)(P.grids[k].Npad + P.grids[k + 1].Npad) * rec_bytes;
        gmax = std::max(gmax, b);
    }
    P.streamed = gmax > budget;
    if (P.streamed && P.form != kF32Recheck)
        return fail(ctx, QT_EUNSUPPORTED,
                    "grids of %zu bytes per layer pair exceed the %zu bytes of shared memory of the plain FP64 form",
                    gmax, budget);
    // samples per thread: tuned value if present, else a register-budget heuristic
    int S = o->tile_samples_per_thread;
    if (S <= 0) S = P.form == kPlainF64 ? 2 : (P.dm <= 2 ? 8 : (P.dm <= 4 ? 4 : 2));
    if (!forward_variant_exists(P.form, P.dm, S, P.streamed))
        return fail(ctx, QT_EUNSUPPORTED, "no kernel for form %d, d %d, %d samples per thread%s", form, d, S,
                    P.streamed ? " (streamed grids)" : "");
    P.S = S;
    P.block = 256;
    P.tile = P.block * S;
    if (P.streamed) {
        long long seg = (long long)(budget / (kSlots * rec_bytes)) / kChunk * kChunk;
        seg = std::min<long long>(seg, 2048);
        if (seg < kChunk) return fail(ctx, QT_EUNSUPPORTED, "records too large for the streamed ring");
        P.seg_records = (int)seg;
        P.grid_bytes = round_up((long long)(kSlots * seg * rec_bytes), 128);
    } else {
        P.grid_bytes = round_up((long long)gmax, 128);
    }
    const bool force_smem = (o->flags & QT_FLAG_SMEM_HIST) != 0;
    const bool force_glob = (o->flags & QT_FLAG_GLOBAL_HIST) != 0;
    size_t hmax = 0;
    P.layers.resize(n);
    long long item = 0, coff = 0;
    const long long items_per_layer = (M + P.tile - 1) / P.tile;
    for (int k = 0; k < n; ++k) {
        LayerDesc& L = P.layers[k];
        memset(&L, 0, sizeof L);
        L.NA = (int)Ns[k];
        L.NB = (int)Ns[k + 1];
        L.NApad = P.grids[k].Npad;
        L.NBpad = P.grids[k + 1].Npad;
        L.gridA = k;
        L.gridB = k + 1;
        L.goffA = P.grids[k].goff;
        L.goffB = P.grids[k + 1].goff;
        L.roffA = P.grids[k].roff;
        L.roffB = P.grids[k + 1].roff;
        L.coff = coff;
        L.item_begin = item;
        L.items = (int)items_per_layer;
        const size_t hb = (size_t)L.NA * L.NB * 4;
        // privatise when the histogram fits and each CTA sees enough samples of
        // the layer to amortise the flush (or when forced)
        const long long ctas = (long long)ctx->num_sms * 2;
        const bool dense_enough = (M / std::max<long long>(ctas, 1)) >= 2 * (long long)L.NA * L.NB;
        L.hist_smem = !P.streamed && !force_glob && hb + P.grid_bytes <= budget && (force_smem || dense_enough);
        if (P.streamed) {
            L.segA = (int)((L.NApad + P.seg_records - 1) / P.seg_records);
            L.segB = (int)((L.NBpad + P.seg_records - 1) / P.seg_records);
        }
        if (L.hist_smem) hmax = std::max(hmax, hb);
        item += items_per_layer;
        coff += (long long)L.NA * L.NB;
    }
    P.total_items = item;
    P.count_entries = coff;
    P.hist_bytes = round_up((long long)hmax, 16);
    P.dyn_smem = P.grid_bytes + P.hist_bytes;
    return QT_OK;
}

bool stream_is_capturing(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// Enqueue the whole forward step on `st`: table uploads, zeroing, record
// preparation, the persistent kernel.
qt_status enqueue_forward(qt_ctx* ctx, const Plan& P, const FwdIO& io, long long M, unsigned long long seed,
                          const qt_options* o, int source, void* dparams_f, void* dparams_d, const void* hparams_f,
                          const void* hparams_d, size_t pcount, void* dlayers, void* dgrids, const void* hlayers,
                          const void* hgrids, void* drec32, void* drec64, DevStatus* dstatus, cudaStream_t st,
                          void* dtiles, void* dtcitems)
{
    QT_CUDA(cudaMemcpyAsync(dparams_f, hparams_f, pcount * 4, cudaMemcpyHostToDevice, st));
    QT_CUDA(cudaMemcpyAsync(dparams_d, hparams_d, pcount * 8, cudaMemcpyHostToDevice, st));
    QT_CUDA(cudaMemcpyAsync(dlayers, hlayers, sizeof(LayerDesc) * P.layers.size(), cudaMemcpyHostToDevice, st));
    QT_CUDA(cudaMemcpyAsync(dgrids, hgrids, sizeof(GridInfo) * P.grids.size(), cudaMemcpyHostToDevice, st));
    QT_CUDA(cudaMemsetAsync(dstatus, 0, sizeof(DevStatus), st));
    const size_t csize = o->counts_type == QT_COUNTS_U32 ? 4 : 8;
    QT_CUDA(cudaMemsetAsync(io.counts, 0, csize * (size_t)P.count_entries, st));
    if (io.dump && io.dump->count > 0) {
        QT_CUDA(cudaMemsetAsync(io.dump->i, 0xFF, sizeof(int32_t) * (size_t)io.dump->count * P.n, st));
        QT_CUDA(cudaMemsetAsync(io.dump->j, 0xFF, sizeof(int32_t) * (size_t)io.dump->count * P.n, st));
    }
    {
        const int blk = 256;
        const long long nb = (P.total_recs + blk - 1) / blk;
        prep_records_kernel<<<(unsigned)nb, blk, 0, st>>>(
            io.g64, (GridInfo*)dgrids, P.ngrids, P.d, P.rec_floats, P.rec64, P.total_recs,
            P.form != kPlainF64 ? (float*)drec32 : nullptr, P.form == kPlainF64 ? (double*)drec64 : nullptr);
        QT_CUDA(cudaGetLastError());
    }
    if (P.form == kTcRecheck) {
        const long long rows = P.tc_total_tiles * kTcTileN;
        prep_tc_tiles_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(
            (const float*)drec32, (GridInfo*)dgrids, P.ngrids, P.d, P.dm, P.rec_floats, P.tc_k, rows, (__half*)dtiles);
        QT_CUDA(cudaGetLastError());
    }
    ForwardParams fp;
    memset(&fp, 0, sizeof fp);
    fp.tc_tiles = dtiles;
    fp.tc_k = P.tc_k;
    fp.tc_slots = P.tc_slots;
    fp.tc_resident = P.tc_resident;
    fp.d = P.d;
    fp.n = P.n;
    fp.form = P.form;
    fp.source = source;
    fp.prec = o->sample_prec == QT_PREC_F32 ? 1 : 0;
    fp.counts_u32 = o->counts_type == QT_COUNTS_U32;
    fp.M = (unsigned long long)M;
    fp.seed = seed;
    fp.total_items = P.total_items;
    fp.tile = P.tile;
    fp.rec_floats = P.rec_floats;
    fp.rec64_doubles = P.rec64;
    fp.smem_grid_bytes = (int)P.grid_bytes;
    fp.smem_hist_entries = (int)(P.hist_bytes / 4);
    fp.seg_records = P.seg_records;
    fp.spin_budget = o->spin_budget == 0 ? 10000000ll : o->spin_budget;   // microseconds (10 s default)
    fp.pathwise_euler = P.euler;
    fp.layers = (const LayerDesc*)dlayers;
    fp.grids = (const GridInfo*)dgrids;
    fp.params_f = (const float*)dparams_f;
    fp.params_d = (const double*)dparams_d;
    fp.params_stride = P.pstride;
    fp.g64 = io.g64;
    fp.rec32 = (const float*)drec32;
    fp.rec64 = (const double*)drec64;
    fp.srcX = io.srcX;
    fp.srcY = io.srcY;
    fp.counts = io.counts;
    fp.cellsA = io.cellsA;
    fp.cellsB = io.cellsB;
    if (io.dump && io.dump->count > 0) {
        fp.dump_count = io.dump->count;
        fp.dump_stride = io.dump->stride;
        fp.dumpX = io.dump->X;
        fp.dumpY = io.dump->Y;
        fp.dumpI = io.dump->i;
        fp.dumpJ = io.dump->j;
    }
    fp.status = dstatus;
    if (P.form == kRouterCert) {
        router_fill_params(static_cast<const qt_router*>(o->router), fp);
        long long pts = 0;
        for (const GridInfo& G : P.grids) pts += G.N;
        cudaError_t ce = launch_grid_checksum(io.g64, pts * P.d, &dstatus->spare[0], st);
        if (ce != cudaSuccess) return fail(ctx, QT_ECUDA, "grid checksum: %s", cudaGetErrorString(ce));
    }
    int blocks_per_sm = 0;
    int launches = 1 + (P.form == kTcRecheck ? 1 : 0) + (P.form == kRouterCert ? 1 : 0);   // preparation
    // timing events around the kernel; inside a capture they must be external
    // event nodes to be recorded at every replay
    const unsigned evflags = stream_is_capturing(st) ? cudaEventRecordExternal : cudaEventRecordDefault;
    QT_CUDA(cudaEventRecordWithFlags(ctx->ev_k0, st, evflags));
    if (P.form == kTcRecheck) {
        // one launch over every work item (or one per window when capped); with
        // the draw-pass layout each window's samples are drawn first
        fp.tc_draw_in = P.tc_draw_in;
        fp.tc_items = (unsigned char*)dtcitems;
        for (long long lo = 0; lo < P.total_items; lo += P.tc_chunk_items) {
            fp.item_lo = lo;
            fp.item_hi = std::min(P.total_items, lo + P.tc_chunk_items);
            cudaError_t e = cudaSuccess;
            if (!P.tc_draw_in) {
                e = launch_tc_draw(P.dm, fp, st);
                if (e != cudaSuccess) return fail(ctx, QT_ECUDA, "draw pass launch: %s", cudaGetErrorString(e));
            }
            e = forward_launch(P.form, P.dm, P.S, P.streamed, fp, P.block, (int)P.dyn_smem, ctx->num_sms,
                               &blocks_per_sm, st);
            launches += P.tc_draw_in ? 1 : 2;
            if (e != cudaSuccess) return fail(ctx, QT_ECUDA, "forward kernel launch: %s", cudaGetErrorString(e));
        }
    } else {
        cudaError_t e = forward_launch(P.form, P.dm, P.S, P.streamed, fp, P.block, (int)P.dyn_smem, ctx->num_sms,
                                       &blocks_per_sm, st);
        if (e != cudaSuccess) return fail(ctx, QT_ECUDA, "forward kernel launch: %s", cudaGetErrorString(e));
    }
    if (P.form != kTcRecheck) ++launches;
    QT_CUDA(cudaEventRecordWithFlags(ctx->ev_k1, st, evflags));
    ctx->timed = true;
    ctx->last_launches = launches;
    ctx->last_tc_draw = P.form == kTcRecheck ? (P.tc_draw_in ? 2 : 1) : 0;
    return QT_OK;
}

qt_status read_status(qt_ctx* ctx, cudaStream_t st, qt_stats* stats, long long samples, long long searches)
{
    void* dstatus = ctx->status_buf;
    DevStatus hs;
    memset(&hs, 0, sizeof hs);
    QT_CUDA(cudaStreamSynchronize(st));
    if (dstatus) QT_CUDA(cudaMemcpy(&hs, dstatus, sizeof hs, cudaMemcpyDeviceToHost));
    if (stats) {
        stats->samples = samples;
        stats->searches = searches;
        stats->rechecks = (int64_t)hs.rechecks;
        stats->candidates = (int64_t)hs.candidates;
        stats->form_used = ctx->last_form;
        stats->launches = ctx->last_launches;
        stats->tc_draw = ctx->last_tc_draw;
        stats->device_status = hs.code;
        stats->ms = 0.0;
        for (int q = 0; q < 3; ++q) stats->diag[q] = (int64_t)hs.spare[q + 1] - (q == 0 ? 0 : 0);
        float ms = 0.f;
        if (ctx->timed && cudaEventElapsedTime(&ms, ctx->ev_k0, ctx->ev_k1) == cudaSuccess) stats->ms = ms;
        cudaGetLastError();
    }
    if (hs.code == QT_ETIMEOUT) return fail(ctx, QT_ETIMEOUT, "a bounded device wait ran out (site %d)", hs.where);
    if (hs.code == QT_EINVAL) return fail(ctx, QT_EINVAL, "the grids differ from those the router was built for");
    if (hs.code != 0) return fail(ctx, QT_EDEVICE, "kernel reported status %d at site %d", hs.code, hs.where);
    return QT_OK;
}

void key_append(std::vector<unsigned char>& k, const void* p, size_t n)
{
    const unsigned char* b = (const unsigned char*)p;
    k.insert(k.end(), b, b + n);
}

// Upload the tables of plan P and run it on `st`, directly or through the
// cached CUDA graph.  `tag` prefixes the workspace names (the autotuner keeps
// its own buffers so that it never invalidates the cached graph).
qt_status run_plan(qt_ctx* ctx, const Plan& P, const FwdIO& io, long long M, unsigned long long seed,
                   const qt_options* o, int source, const double* params_d_host, cudaStream_t st, bool use_graph,
                   const std::string& tag)
{
    qt_status s;
    const int n = P.n;
    void *dlayers, *dgrids, *dpf, *dpd, *drec32 = nullptr, *drec64 = nullptr, *dstatus;
    const size_t pbytes = (size_t)std::max(1, n) * P.pstride;
    if ((s = dev_get(ctx, (tag + "layers").c_str(), sizeof(LayerDesc) * P.layers.size(), &dlayers))) return s;
    if ((s = dev_get(ctx, (tag + "grids").c_str(), sizeof(GridInfo) * P.grids.size(), &dgrids))) return s;
    if ((s = dev_get(ctx, (tag + "params_f").c_str(), pbytes * 4, &dpf))) return s;
    if ((s = dev_get(ctx, (tag + "params_d").c_str(), pbytes * 8, &dpd))) return s;
    if (P.form != kPlainF64) {
        if ((s = dev_get(ctx, (tag + "rec32").c_str(), (size_t)P.total_recs * P.rec_floats * 4, &drec32))) return s;
    } else {
        if ((s = dev_get(ctx, (tag + "rec64").c_str(), (size_t)P.total_recs * P.rec64 * 8, &drec64))) return s;
    }
    if ((s = dev_get(ctx, (tag + "status").c_str(), sizeof(DevStatus), &dstatus))) return s;
    void* dtiles = nullptr;
    void* dtcitems = nullptr;
    if (P.form == kTcRecheck &&
        ((s = dev_get(ctx, (tag + "tctiles").c_str(), (size_t)P.tc_total_tiles * kTcTileN * P.tc_k * 2, &dtiles)) ||
         (!P.tc_draw_in &&
          (s = dev_get(ctx, (tag + "tcitems").c_str(), (size_t)P.tc_chunk_items * P.tc_item_bytes, &dtcitems)))))
        return s;
    void *hlayers, *hgrids, *hpf, *hpd;
    if ((s = host_get(ctx, (tag + "layers").c_str(), sizeof(LayerDesc) * P.layers.size(), &hlayers))) return s;
    if ((s = host_get(ctx, (tag + "grids").c_str(), sizeof(GridInfo) * P.grids.size(), &hgrids))) return s;
    if ((s = host_get(ctx, (tag + "params_f").c_str(), pbytes * 4, &hpf))) return s;
    if ((s = host_get(ctx, (tag + "params_d").c_str(), pbytes * 8, &hpd))) return s;
    // the previous replay may still read the pinned tables
    QT_CUDA(cudaEventSynchronize(ctx->ev_tables));
    memcpy(hlayers, P.layers.data(), sizeof(LayerDesc) * P.layers.size());
    memcpy(hgrids, P.grids.data(), sizeof(GridInfo) * P.grids.size());
    float* pf = (float*)hpf;
    double* pd = (double*)hpd;
    memset(pf, 0, pbytes * 4);
    memset(pd, 0, pbytes * 8);
    if (params_d_host) {
        for (long long e = 0; e < (long long)n * P.pstride; ++e) {
            pd[e] = params_d_host[e];
            pf[e] = (float)params_d_host[e];
        }
    }
    ctx->status_buf = dstatus;
    if (!use_graph) {
        s = enqueue_forward(ctx, P, io, M, seed, o, source, dpf, dpd, hpf, hpd, pbytes, dlayers, dgrids, hlayers,
                            hgrids, drec32, drec64, (DevStatus*)dstatus, st, dtiles, dtcitems);
        if (s) return s;
    } else {
        // graph key: everything the enqueued work depends on
        std::vector<unsigned char> key;
        key_append(key, &P.form, sizeof P.form);
        key_append(key, &P.S, sizeof P.S);
        key_append(key, &P.streamed, sizeof P.streamed);
        key_append(key, &P.seg_records, sizeof P.seg_records);
        key_append(key, &P.euler, sizeof P.euler);
        key_append(key, &M, sizeof M);
        key_append(key, &seed, sizeof seed);
        key_append(key, &source, sizeof source);
        key_append(key, o, sizeof *o);
        key_append(key, &io, sizeof io);
        if (io.dump) key_append(key, io.dump, sizeof *io.dump);
        key_append(key, P.layers.data(), sizeof(LayerDesc) * P.layers.size());
        key_append(key, P.grids.data(), sizeof(GridInfo) * P.grids.size());
        key_append(key, pd, pbytes * 8);
        if (!ctx->gexec || key != ctx->gkey) {
            if (ctx->gexec) {
                cudaGraphExecDestroy(ctx->gexec);
                ctx->gexec = nullptr;
            }
            cudaGraph_t graph = nullptr;
            QT_CUDA(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
            qt_status es = enqueue_forward(ctx, P, io, M, seed, o, source, dpf, dpd, hpf, hpd, pbytes, dlayers,
                                           dgrids, hlayers, hgrids, drec32, drec64, (DevStatus*)dstatus,
                                           ctx->cap_stream, dtiles, dtcitems);
            cudaError_t ee = cudaStreamEndCapture(ctx->cap_stream, &graph);
            if (es != QT_OK || ee != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                if (es != QT_OK) return es;
                return fail(ctx, QT_ECUDA, "graph capture: %s", cudaGetErrorString(ee));
            }
            cudaError_t ie = cudaGraphInstantiate(&ctx->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) {
                ctx->gexec = nullptr;
                return fail(ctx, QT_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
            }
            ctx->gkey = key;
        }
        QT_CUDA(cudaGraphLaunch(ctx->gexec, st));
    }
    QT_CUDA(cudaEventRecord(ctx->ev_tables, st));
    return QT_OK;
}

// Autotuner: time every compiled samples-per-thread variant of this problem's
// kernel class on a probe (first layers, bounded M) and keep the fastest for
// the (form, mode, dimension class, precision, grid-size class) key.
qt_status autotune(qt_ctx* ctx, int d, int n, const int64_t* Ns, const double* mus, const double* params_d_host,
                   long long M, unsigned long long seed, const qt_options* o, int source, const FwdIO& io,
                   const Plan& base, const TuneKey& key, cudaStream_t st)
{
    static const int cands[] = {1, 2, 4, 8};
    // probe the widest pair of layers (the costliest work items)
    int k0 = 0;
    for (int k = 1; k < n; ++k)
        if (Ns[k] + Ns[k + 1] > Ns[k0] + Ns[k0 + 1]) k0 = k;
    const int n2 = std::min(n - k0, 2);
    Ns += k0;
    mus += (long long)k0 * d;
    if (params_d_host) params_d_host += (long long)k0 * base.pstride;
    const long long M2 = std::min<long long>(M, base.dm <= 4 ? (1ll << 20) : (1ll << 16));
    long long ent = 0;
    for (int k = 0; k < n2; ++k) ent += Ns[k] * Ns[k + 1];
    void* tcounts;
    qt_status s = dev_get(ctx, "tune.counts", (size_t)ent * 8, &tcounts);
    if (s) return s;
    FwdIO tio = io;
    tio.counts = tcounts;
    tio.dump = nullptr;
    tio.cellsA = tio.cellsB = nullptr;
    cudaEvent_t e0, e1;
    QT_CUDA(cudaEventCreate(&e0));
    QT_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int bestS = base.S;
    for (int S : cands) {
        if (!forward_variant_exists(base.form, base.dm, S, base.streamed)) continue;
        qt_options to = *o;
        to.tile_samples_per_thread = S;
        to.counts_type = QT_COUNTS_I64;
        to.flags |= QT_FLAG_NO_TUNE;
        Plan P;
        if (make_plan(ctx, d, n2, Ns, mus, M2, &to, source == kArrays, P) != QT_OK) continue;
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            QT_CUDA(cudaEventRecord(e0, st));
            if ((s = run_plan(ctx, P, tio, M2, seed, &to, source, params_d_host, st, false, "tune."))) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return s;
            }
            QT_CUDA(cudaEventRecord(e1, st));
            QT_CUDA(cudaEventSynchronize(e1));
            QT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        }
        if (ms < best) {
            best = ms;
            bestS = S;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tune[key] = bestS;
    return QT_OK;
}

// Autotuner of the tensor-core form: time both sample-draw layouts (a separate
// draw pass, or the screen kernel drawing its own samples) on the widest window
// of up to four consecutive layer pairs with up to 2^20 samples each (best of
// three runs), keep the faster for the key.
qt_status autotune_tc(qt_ctx* ctx, int d, int n, const int64_t* Ns, const double* mus, const double* params_d_host,
                      long long M, unsigned long long seed, const qt_options* o, int source, const FwdIO& io,
                      const Plan& base, const TuneKey& key, cudaStream_t st)
{
    const int n2 = std::min(n, 4);
    int k0 = 0;
    long long wbest = -1;
    for (int k = 0; k + n2 <= n; ++k) {
        long long w = 0;
        for (int q = k; q < k + n2; ++q) w += Ns[q] + Ns[q + 1];
        if (w > wbest) {
            wbest = w;
            k0 = k;
        }
    }
    Ns += k0;
    mus += (long long)k0 * d;
    if (params_d_host) params_d_host += (long long)k0 * base.pstride;
    const long long M2 = std::min<long long>(M, 1ll << 20);
    long long ent = 0;
    for (int k = 0; k < n2; ++k) ent += Ns[k] * Ns[k + 1];
    void* tcounts;
    qt_status s = dev_get(ctx, "tune.counts", (size_t)ent * 8, &tcounts);
    if (s) return s;
    FwdIO tio = io;
    tio.counts = tcounts;
    tio.dump = nullptr;
    tio.cellsA = tio.cellsB = nullptr;
    cudaEvent_t e0, e1;
    QT_CUDA(cudaEventCreate(&e0));
    QT_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int bestv = 2;
    for (int v = 1; v <= 2; ++v) {
        qt_options to = *o;
        to.tc_draw = v;
        to.tc_chunk_items = 0;
        to.counts_type = QT_COUNTS_I64;
        to.flags |= QT_FLAG_NO_TUNE;
        Plan P;
        if (make_plan(ctx, d, n2, Ns, mus, M2, &to, source == kArrays, P) != QT_OK) continue;
        float fastest = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            QT_CUDA(cudaEventRecord(e0, st));
            if ((s = run_plan(ctx, P, tio, M2, seed, &to, source, params_d_host, st, false, "tune."))) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return s;
            }
            QT_CUDA(cudaEventRecord(e1, st));
            QT_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            QT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) fastest = std::min(fastest, ms);     // the first run warms up
        }
        if (fastest < best) {
            best = fastest;
            bestv = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tune[key] = bestv;
    return QT_OK;
}

TuneKey tune_key(const Plan& P, int prec, const int64_t* Ns, int n)
{
    long long mx = 1;
    for (int k = 0; k <= n; ++k) mx = std::max<long long>(mx, Ns[k]);
    int bucket = 0;
    while ((1ll << bucket) < mx) ++bucket;
    return TuneKey{P.form * 2 + (P.streamed ? 1 : 0), P.dm, prec, bucket};
}

// Shared body of qt_transitions and qt_counts_from_samples.
qt_status forward_common(qt_ctx* ctx, int d, int n, const int64_t* Ns, const double* mus, const double* params_d_host,
                         long long M, unsigned long long seed, const qt_options* o, int source, const FwdIO& io,
                         qt_stats* stats, cudaStream_t st, int only_layer = -1, int algo = 3, int euler = 0)
{
    qt_options oi;
    if (only_layer >= 0 && only_layer == injected_timeout_layer()) {
        oi = *o;
        oi.spin_budget = -1;
        o = &oi;
    }
    Plan P;
    qt_status s = make_plan(ctx, d, n, Ns, mus, M, o, source == kArrays, P, only_layer, algo);
    if (s) return s;
    P.euler = euler;
    const bool capturing = stream_is_capturing(st);
    if (P.form == kTcRecheck && o->tc_draw == 0 && !(o->flags & QT_FLAG_NO_TUNE) && !capturing &&
        o->spin_budget >= 0 && source == kSampler) {
        const TuneKey key = tune_key(P, o->sample_prec, Ns, n);
        if (!ctx->tune.count(key)) {
            if ((s = autotune_tc(ctx, d, n, Ns, mus, params_d_host, M, seed, o, source, io, P, key, st))) return s;
        }
        if (o != &oi) {
            oi = *o;
            o = &oi;
        }
        oi.tc_draw = ctx->tune[key];
        Plan P2;
        if ((s = make_plan(ctx, d, n, Ns, mus, M, o, source == kArrays, P2, only_layer, algo))) return s;
        P2.euler = euler;
        P = P2;
    }
    if (P.form != kTcRecheck && P.form != kRouterCert && P.form != kPathwise && o->tile_samples_per_thread <= 0 &&
        !(o->flags & QT_FLAG_NO_TUNE) && !capturing && o->spin_budget >= 0) {
        const TuneKey key = tune_key(P, source == kArrays ? 0 : o->sample_prec, Ns, n);
        if (!ctx->tune.count(key)) {
            if ((s = autotune(ctx, d, n, Ns, mus, params_d_host, M, seed, o, source, io, P, key, st))) return s;
        }
        qt_options to = *o;
        to.tile_samples_per_thread = ctx->tune[key];
        Plan P2;
        if ((s = make_plan(ctx, d, n, Ns, mus, M, &to, source == kArrays, P2, only_layer))) return s;
        P = P2;
    }
    ctx->last_form = P.form == kPlainF64    ? QT_FORM_PLAIN_F64
                     : P.form == kTcRecheck ? QT_FORM_TC_RECHECK
                     : P.form == kRouterCert ? QT_FORM_ROUTER_CERT
                                             : QT_FORM_F32_RECHECK;
    // one layer at a time (fused backward) launches directly: each layer would be a new graph
    const bool use_graph = !(o->flags & QT_FLAG_NO_GRAPH) && !capturing && only_layer < 0;
    if ((s = run_plan(ctx, P, io, M, seed, o, source, params_d_host, st, use_graph, ""))) return s;
    if (stats) return read_status(ctx, st, stats, (long long)n * M, (algo == 2 ? n + 1ll : 2ll * n) * M);
    return QT_OK;
}

// Pack m, b, L, A, T of layer k (FP64) in the order the sampler reads them,
// then the Euler-scheme scaling alpha, beta (1 and 0 without one).
void pack_params(const qt_model* m, const qt_euler* eu, int k, int pstride, double* out)
{
    const int d = m->d;
    double* p = out + (long long)k * pstride;
    for (int l = 0; l < d; ++l) p[l] = m->m[(long long)k * d + l];
    for (int l = 0; l < d; ++l) p[d + l] = m->b[(long long)k * d + l];
    for (int e = 0; e < d * d; ++e) {
        const int r = e / d, c = e % d;
        p[2 * d + e] = c <= r ? m->L[(long long)k * d * d + e] : 0.0;
        p[2 * d + d * d + e] = m->A[(long long)k * d * d + e];
        p[2 * d + 2 * d * d + e] = c <= r ? m->T[(long long)k * d * d + e] : 0.0;
    }
    for (int l = 0; l < d; ++l) {
        p[2 * d + 3 * d * d + l] = eu ? eu->alpha[(long long)k * d + l] : 1.0;
        p[3 * d + 3 * d * d + l] = eu ? eu->beta[(long long)k * d + l] : 0.0;
    }
}

}  // namespace

namespace {
qt_status transitions_impl(qt_ctx* ctx, const qt_model* model, const double* grids, int64_t M, uint64_t seed,
                           const qt_options* opts, void* counts, const qt_dump* dump, qt_stats* stats, void* stream,
                           int only_layer);
}

extern "C" qt_status qt_transitions(qt_ctx* ctx, const qt_model* model, const double* grids, int64_t M, uint64_t seed,
                                    const qt_options* opts, void* counts, const qt_dump* dump, qt_stats* stats,
                                    void* stream)
{
    return transitions_impl(ctx, model, grids, M, seed, opts, counts, dump, stats, stream, -1);
}

namespace {
// qt_transitions for all layers, or for layer pair `only_layer` alone (its
// counts at the start of `counts`).
qt_status transitions_impl(qt_ctx* ctx, const qt_model* model, const double* grids, int64_t M, uint64_t seed,
                           const qt_options* opts, void* counts, const qt_dump* dump, qt_stats* stats, void* stream,
                           int only_layer)
{
    if (!ctx) return QT_EINVAL;
    qt_status s = validate_model(ctx, model);
    if (s) return s;
    if (!grids || !counts) return fail(ctx, QT_EINVAL, "grids or counts is NULL");
    if (M < 1 || M > 0xFFFFFFFFll) return fail(ctx, QT_EINVAL, "M = %lld outside [1, 2^32)", (long long)M);
    qt_options o;
    if (opts) o = *opts; else qt_default_options(&o);
    if (o.counts_type != QT_COUNTS_I64 && o.counts_type != QT_COUNTS_U32)
        return fail(ctx, QT_EINVAL, "counts_type %d", o.counts_type);
    if (dump && dump->count > 0) {
        if (dump->stride < 1 || !dump->X || !dump->Y || !dump->i || !dump->j)
            return fail(ctx, QT_EINVAL, "dump needs stride >= 1 and four buffers");
    }
    DeviceGuard g(ctx->device);
    const int d = model->d, n = model->n;
    const int pstride = param_stride(d);
    std::vector<double> params((size_t)n * pstride, 0.0);
    for (int k = 0; k < n; ++k) pack_params(model, nullptr, k, pstride, params.data());
    FwdIO io;
    memset(&io, 0, sizeof io);
    io.g64 = grids;
    io.counts = counts;
    io.dump = (dump && dump->count > 0) ? dump : nullptr;
    return forward_common(ctx, d, n, model->N, model->m, params.data(), M, seed, &o, kSampler, io, stats,
                          (cudaStream_t)stream, only_layer);
}
}  // namespace

extern "C" qt_status qt_transitions_pathwise(qt_ctx* ctx, const qt_model* model, const qt_euler* euler,
                                             const double* grids, int64_t M, uint64_t seed, const qt_options* opts,
                                             void* counts, const qt_dump* dump, qt_stats* stats, void* stream)
{
    if (!ctx) return QT_EINVAL;
    qt_status s = validate_model(ctx, model);
    if (s) return s;
    if (!grids || !counts) return fail(ctx, QT_EINVAL, "grids or counts is NULL");
    if (M < 1 || M > 0xFFFFFFFFll) return fail(ctx, QT_EINVAL, "M = %lld outside [1, 2^32)", (long long)M);
    if (euler && (!euler->alpha || !euler->beta)) return fail(ctx, QT_EINVAL, "euler needs alpha and beta");
    qt_options o;
    if (opts) o = *opts; else qt_default_options(&o);
    if (o.counts_type != QT_COUNTS_I64 && o.counts_type != QT_COUNTS_U32)
        return fail(ctx, QT_EINVAL, "counts_type %d", o.counts_type);
    if (o.sample_prec != QT_PREC_F32 && o.sample_prec != QT_PREC_F64)
        return fail(ctx, QT_EINVAL, "sample_prec %d", o.sample_prec);
    if (dump && dump->count > 0) {
        if (dump->stride < 1 || !dump->X || !dump->Y || !dump->i || !dump->j)
            return fail(ctx, QT_EINVAL, "dump needs stride >= 1 and four buffers");
    }
    DeviceGuard g(ctx->device);
    const int d = model->d, n = model->n;
    const int pstride = param_stride(d);
    std::vector<double> params((size_t)n * pstride, 0.0);
    for (int k = 0; k < n; ++k) pack_params(model, euler, k, pstride, params.data());
    FwdIO io;
    memset(&io, 0, sizeof io);
    io.g64 = grids;
    io.counts = counts;
    io.dump = (dump && dump->count > 0) ? dump : nullptr;
    return forward_common(ctx, d, n, model->N, model->m, params.data(), M, seed, &o, kSampler, io, stats,
                          (cudaStream_t)stream, -1, 2, euler ? 1 : 0);
}

extern "C" qt_status qt_counts_from_samples(qt_ctx* ctx, int32_t d, const double* gA, int64_t NA, const double* gB,
                                            int64_t NB, const double* X, const double* Y, int64_t M,
                                            const qt_options* opts, void* counts, int32_t* ii, int32_t* jj,
                                            qt_stats* stats, void* stream)
{
    if (!ctx) return QT_EINVAL;
    if (d < 1 || d > kDMax) return fail(ctx, QT_EINVAL, "d = %d outside [1, %d]", d, kDMax);
    if (!gA || !gB || !X || !Y || !counts) return fail(ctx, QT_EINVAL, "NULL array");
    if (NA < 1 || NB < 1 || NA > (1 << 24) || NB > (1 << 24)) return fail(ctx, QT_EINVAL, "grid sizes");
    if (M < 1 || M > 0xFFFFFFFFll) return fail(ctx, QT_EINVAL, "M = %lld outside [1, 2^32)", (long long)M);
    if ((ii == nullptr) != (jj == nullptr)) return fail(ctx, QT_EINVAL, "ii and jj must both be set or both NULL");
    qt_options o;
    if (opts) o = *opts; else qt_default_options(&o);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    // both grids contiguous in one workspace buffer
    void* dg;
    qt_status s = dev_get(ctx, "pair_grids", sizeof(double) * (size_t)(NA + NB) * d, &dg);
    if (s) return s;
    QT_CUDA(cudaMemcpyAsync(dg, gA, sizeof(double) * NA * d, cudaMemcpyDeviceToDevice, st));
    QT_CUDA(cudaMemcpyAsync((double*)dg + NA * d, gB, sizeof(double) * NB * d, cudaMemcpyDeviceToDevice, st));
    // centres of the screen: zero (the bound uses the norms about this centre)
    std::vector<double> mus((size_t)2 * d, 0.0);
    int64_t Ns[2] = {NA, NB};
    FwdIO io;
    memset(&io, 0, sizeof io);
    io.g64 = (const double*)dg;
    io.counts = counts;
    io.srcX = X;
    io.srcY = Y;
    io.cellsA = ii;
    io.cellsB = jj;
    o.sample_prec = QT_PREC_F64;
    o.flags |= QT_FLAG_NO_GRAPH;
    return forward_common(ctx, d, 1, Ns, mus.data(), nullptr, M, 0, &o, kArrays, io, stats, st);
}

extern "C" qt_status qt_get_status(qt_ctx* ctx, void* stream, qt_stats* stats)
{
    if (!ctx) return QT_EINVAL;
    DeviceGuard g(ctx->device);
    return read_status(ctx, (cudaStream_t)stream, stats, 0, 0);
}

extern "C" qt_status qt_transitions_workspace(const qt_model* model, const qt_options* opts, size_t* bytes)
{
    if (!model || !bytes || model->d < 1 || model->d > kDMax || model->n < 1) return QT_EINVAL;
    qt_options o;
    if (opts) o = *opts; else qt_default_options(&o);
    const int d = model->d, n = model->n, dm = dm_for(d);
    long long recs = 0;
    for (int k = 0; k <= n; ++k) recs += round_up(model->N[k], kChunk);
    const long long pstride = param_stride(d);
    size_t b = sizeof(LayerDesc) * n + sizeof(GridInfo) * (n + 1) + (size_t)n * pstride * 12 + sizeof(DevStatus);
    b += o.form == QT_FORM_PLAIN_F64 ? (size_t)recs * rec64_for(dm) * 8 : (size_t)recs * rec_floats_for(dm) * 4;
    *bytes = b;
    return QT_OK;
}

// ------------------------------------------------------------------ backward induction and price

extern "C" qt_status qt_backward(qt_ctx* ctx, int32_t n, const int64_t* N, const void* counts, int32_t counts_type,
                                 const double* phi, double* V, void* stream)
{
    if (!ctx) return QT_EINVAL;
    if (n < 1 || !N || !counts || !phi || !V) return fail(ctx, QT_EINVAL, "bad arguments to qt_backward");
    if (counts_type != QT_COUNTS_I64 && counts_type != QT_COUNTS_U32)
        return fail(ctx, QT_EINVAL, "counts_type %d", counts_type);
    for (int k = 0; k <= n; ++k)
        if (N[k] < 1 || N[k] > (1 << 24)) return fail(ctx, QT_EINVAL, "N[%d]", k);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<long long> goff(n + 2, 0), coff(n + 1, 0);
    for (int k = 0; k <= n; ++k) goff[k + 1] = goff[k] + N[k];
    for (int k = 0; k < n; ++k) coff[k + 1] = coff[k] + N[k] * N[k + 1];
    QT_CUDA(cudaMemcpyAsync(V + goff[n], phi + goff[n], sizeof(double) * N[n], cudaMemcpyDeviceToDevice, st));
    const int u32 = counts_type == QT_COUNTS_U32;
    for (int k = n - 1; k >= 0; --k) {
        const long long threads = (long long)N[k] * 32;
        const int blk = 256;
        backward_layer_kernel<<<(unsigned)((threads + blk - 1) / blk), blk, 0, st>>>(
            counts, u32, coff[k], (int)N[k], (int)N[k + 1], phi + goff[k], V + goff[k + 1], V + goff[k]);
        QT_CUDA(cudaGetLastError());
    }
    return QT_OK;
}

extern "C" qt_status qt_swing(qt_ctx* ctx, int32_t n, const int64_t* N, const void* counts, int32_t counts_type,
                              const double* v, int32_t Qmin, int32_t Qmax, double* P, double* price, void* stream)
{
    if (!ctx) return QT_EINVAL;
    if (n < 1 || !N || !counts || !v || !P) return fail(ctx, QT_EINVAL, "bad arguments to qt_swing");
    if (counts_type != QT_COUNTS_I64 && counts_type != QT_COUNTS_U32)
        return fail(ctx, QT_EINVAL, "counts_type %d", counts_type);
    if (Qmin < 0 || Qmax < Qmin || Qmin > n || Qmax > (1 << 20))
        return fail(ctx, QT_EINVAL, "volume constraint [%d, %d] with n = %d", Qmin, Qmax, n);
    for (int k = 0; k <= n; ++k)
        if (N[k] < 1 || N[k] > (1 << 24)) return fail(ctx, QT_EINVAL, "N[%d]", k);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const long long nq = (long long)Qmax + 1;
    std::vector<long long> goff(n + 2, 0), coff(n + 1, 0);
    for (int k = 0; k <= n; ++k) goff[k + 1] = goff[k] + N[k];
    for (int k = 0; k < n; ++k) coff[k + 1] = coff[k] + N[k] * N[k + 1];
    const long long tn = nq * N[n];
    swing_terminal_kernel<<<(unsigned)((tn + 255) / 256), 256, 0, st>>>((int)N[n], n, Qmin, Qmax, P + nq * goff[n]);
    QT_CUDA(cudaGetLastError());
    const int u32 = counts_type == QT_COUNTS_U32;
    const long long qchunks = (Qmax + kSwingQ) / kSwingQ;   // warps per grid row
    for (int k = 0; k < n; ++k)
        if ((N[k] * qchunks * 32 + 255) / 256 > 0x7FFFFFFFll)
            return fail(ctx, QT_EINVAL, "N[%d] x (Qmax + 1) too large for one launch", k);
    for (int k = n - 1; k >= 0; --k) {
        const long long threads = (long long)N[k] * qchunks * 32;
        swing_layer_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
            counts, u32, coff[k], (int)N[k], (int)N[k + 1], v + goff[k], P + nq * goff[k + 1], P + nq * goff[k], n,
            k, Qmin, Qmax);
        QT_CUDA(cudaGetLastError());
    }
    if (price) {
        void* dout;
        qt_status s = dev_get(ctx, "swing_out", sizeof(double), &dout);
        if (s) return s;
        root_price_kernel<<<1, 32, 0, st>>>(counts, u32, (int)N[0], (int)N[1], P, (double*)dout);
        QT_CUDA(cudaGetLastError());
        QT_CUDA(cudaMemcpyAsync(price, dout, sizeof(double), cudaMemcpyDeviceToHost, st));
        QT_CUDA(cudaStreamSynchronize(st));
    }
    return QT_OK;
}

namespace {
bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace

extern "C" qt_status qt_price(qt_ctx* ctx, const qt_model* model, const double* grids, int64_t M, uint64_t seed,
                              const qt_options* opts, const double* phi, double* price, qt_stats* stats, void* stream)
{
    if (!ctx) return QT_EINVAL;
    qt_status s = validate_model(ctx, model);
    if (s) return s;
    if (!grids || !phi || !price) return fail(ctx, QT_EINVAL, "NULL argument to qt_price");
    qt_options o;
    if (opts) o = *opts; else qt_default_options(&o);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int n = model->n, d = model->d;
    long long pts = 0, ent = 0;
    for (int k = 0; k <= n; ++k) pts += model->N[k];
    for (int k = 0; k < n; ++k) ent += model->N[k] * model->N[k + 1];
    const size_t csize = o.counts_type == QT_COUNTS_U32 ? 4 : 8;
    const bool fused = (o.flags & QT_FLAG_FUSED_BACKWARD) != 0;
    if (fused) {
        // one layer's counts at a time
        ent = 0;
        for (int k = 0; k < n; ++k) ent = std::max<long long>(ent, model->N[k] * model->N[k + 1]);
    }
    void *dcounts, *dV, *dout;
    if ((s = dev_get(ctx, "price_counts", csize * (size_t)ent, &dcounts))) return s;
    if ((s = dev_get(ctx, "price_V", sizeof(double) * (size_t)pts, &dV))) return s;
    if ((s = dev_get(ctx, "price_out", sizeof(double), &dout))) return s;
    const double* dgrids = grids;
    const double* dphi = phi;
    if (!is_device_ptr(grids)) {
        void* p;
        if ((s = dev_get(ctx, "price_grids", sizeof(double) * (size_t)pts * d, &p))) return s;
        QT_CUDA(cudaMemcpyAsync(p, grids, sizeof(double) * (size_t)pts * d, cudaMemcpyHostToDevice, st));
        dgrids = (const double*)p;
    }
    if (!is_device_ptr(phi)) {
        void* p;
        if ((s = dev_get(ctx, "price_phi", sizeof(double) * (size_t)pts, &p))) return s;
        QT_CUDA(cudaMemcpyAsync(p, phi, sizeof(double) * (size_t)pts, cudaMemcpyHostToDevice, st));
        dphi = (const double*)p;
    }
    if (!fused) {
        if ((s = qt_transitions(ctx, model, dgrids, M, seed, &o, dcounts, nullptr, nullptr, stream))) return s;
        if ((s = qt_backward(ctx, n, model->N, dcounts, o.counts_type, dphi, (double*)dV, stream))) return s;
    } else {
        // layers in reverse order: the counts of pair (k, k + 1), then V_k from
        // them and V_{k+1} at once (the same kernels and arithmetic as the
        // unfused path, so the same bits); the counts left at the end are
        // layer 0's, which the root value reads
        std::vector<long long> goff(n + 2, 0);
        for (int k = 0; k <= n; ++k) goff[k + 1] = goff[k] + model->N[k];
        double* V = (double*)dV;
        // each layer's launch clears its own status block: fold every one into
        // an accumulator, so that an error in any layer reaches the caller
        void* dacc;
        if ((s = dev_get(ctx, "price_status", sizeof(DevStatus), &dacc))) return s;
        QT_CUDA(cudaMemsetAsync(dacc, 0, sizeof(DevStatus), st));
        QT_CUDA(cudaMemcpyAsync(V + goff[n], dphi + goff[n], sizeof(double) * model->N[n], cudaMemcpyDeviceToDevice,
                                st));
        for (int k = n - 1; k >= 0; --k) {
            if ((s = transitions_impl(ctx, model, dgrids, M, seed, &o, dcounts, nullptr, nullptr, stream, k)))
                return s;
            fold_status_kernel<<<1, 1, 0, st>>>((const DevStatus*)ctx->status_buf, (DevStatus*)dacc);
            QT_CUDA(cudaGetLastError());
            const long long threads = model->N[k] * 32;
            backward_layer_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
                dcounts, o.counts_type == QT_COUNTS_U32, 0, (int)model->N[k], (int)model->N[k + 1], dphi + goff[k],
                V + goff[k + 1], V + goff[k]);
            QT_CUDA(cudaGetLastError());
        }
        // the status the caller reads is the accumulated one
        QT_CUDA(cudaMemcpyAsync(ctx->status_buf, dacc, sizeof(DevStatus), cudaMemcpyDeviceToDevice, st));
    }
    root_price_kernel<<<1, 32, 0, st>>>(dcounts, o.counts_type == QT_COUNTS_U32, (int)model->N[0], (int)model->N[1],
                                        (const double*)dV, (double*)dout);
    QT_CUDA(cudaGetLastError());
    QT_CUDA(cudaMemcpyAsync(price, dout, sizeof(double), cudaMemcpyDeviceToHost, st));
    return read_status(ctx, st, stats, (long long)n * M, 2ll * n * M);
}

// ------------------------------------------------------------------ grid builder

namespace {

double npdf(double z) { return std::isfinite(z) ? std::exp(-0.5 * z * z) * 0.3989422804014327 : 0.0; }
double ncdf_upper(double z) { return 0.5 * std::erfc(z * 0.7071067811865476); }   // P(Z > z)
double cell_mass(double lo, double hi)
{
    return hi <= 0 ? ncdf_upper(-hi) - ncdf_upper(-lo) : ncdf_upper(lo) - ncdf_upper(hi);
}

// Stationary N-point quantizer of N(0,1): Lloyd's map on closed-form cell
// means, then Newton on G_i = x_i P_i - (pdf(b_{i-1}) - pdf(b_i)) (tridiagonal).
std::vector<double> lloyd1d(int N, double tol)
{
    std::vector<double> x(N, 0.0);
    if (N == 1) return x;
    // quantile start via bisection on the upper tail
    for (int i = 0; i < N; ++i) {
        const double p = (i + 0.5) / N;
        double lo = -10, hi = 10;
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (1.0 - ncdf_upper(mid) < p) lo = mid; else hi = mid;
        }
        x[i] = 0.5 * (lo + hi);
    }
    std::vector<double> lo(N), hi(N), P(N), Q(N), G(N), a(N), b(N), c(N), step(N);
    auto cells = [&]() {
        for (int i = 0; i < N; ++i) {
            lo[i] = i == 0 ? -INFINITY : 0.5 * (x[i - 1] + x[i]);
            hi[i] = i == N - 1 ? INFINITY : 0.5 * (x[i] + x[i + 1]);
            P[i] = cell_mass(lo[i], hi[i]);
            Q[i] = npdf(lo[i]) - npdf(hi[i]);
        }
    };
    for (int it = 0; it < 200; ++it) {
        cells();
        for (int i = 0; i < N; ++i) x[i] = Q[i] / P[i];
    }
    for (int it = 0; it < 100; ++it) {
        cells();
        for (int i = 0; i < N; ++i) {
            G[i] = x[i] * P[i] - Q[i];
            const double lf = std::isfinite(lo[i]) ? lo[i] : 0.0, hf = std::isfinite(hi[i]) ? hi[i] : 0.0;
            b[i] = P[i] + 0.5 * (x[i] - hf) * npdf(hi[i]) + 0.5 * (lf - x[i]) * npdf(lo[i]);
            c[i] = i < N - 1 ? 0.5 * (x[i] - hf) * npdf(hi[i]) : 0.0;
            a[i] = i > 0 ? 0.5 * (lf - x[i]) * npdf(lo[i]) : 0.0;
        }
        // Thomas algorithm
        std::vector<double> cp(N), dp(N);
        cp[0] = c[0] / b[0];
        dp[0] = G[0] / b[0];
        for (int i = 1; i < N; ++i) {
            const double den = b[i] - a[i] * cp[i - 1];
            cp[i] = c[i] / den;
            dp[i] = (G[i] - a[i] * dp[i - 1]) / den;
        }
        step[N - 1] = dp[N - 1];
        for (int i = N - 2; i >= 0; --i) step[i] = dp[i] - cp[i] * step[i + 1];
        double mx = 0;
        for (int i = 0; i < N; ++i) {
            x[i] -= step[i];
            mx = std::max(mx, std::fabs(step[i]));
        }
        for (int i = 0; i < N / 2; ++i) {  // exact symmetry of the optimum
            const double v = 0.5 * (x[N - 1 - i] - x[i]);
            x[i] = -v;
            x[N - 1 - i] = v;
        }
        if (N % 2) x[N / 2] = 0.0;
        if (mx < tol) break;
    }
    return x;
}

void factor_sizes(int N, int d, std::vector<int>& best, std::vector<int>& cur, double& score)
{
    if (d == 1) {
        cur.push_back(N);
        int mx = *std::max_element(cur.begin(), cur.end()), mn = *std::min_element(cur.begin(), cur.end());
        const double sc = (double)mx / mn;
        if (best.empty() || sc < score) {
            score = sc;
            best = cur;
        }
        cur.pop_back();
        return;
    }
    for (int a = 1; a <= N; ++a) {
        if (N % a) continue;
        cur.push_back(a);
        factor_sizes(N / a, d - 1, best, cur, score);
        cur.pop_back();
    }
}

}  // namespace

extern "C" qt_status qt_build_grids(qt_ctx* ctx, const qt_model* model, int32_t method, int64_t samples, int32_t iters,
                                    double tol, uint64_t seed, double* grids, void* stream)
{
    if (!ctx) return QT_EINVAL;
    qt_status s = validate_model(ctx, model);
    if (s) return s;
    if (!grids) return fail(ctx, QT_EINVAL, "grids is NULL");
    const int d = model->d, n = model->n;
    if (method == QT_GRID_LLOYD1D && d != 1) return fail(ctx, QT_EINVAL, "QT_GRID_LLOYD1D needs d = 1");
    if (method != QT_GRID_LLOYD1D && method != QT_GRID_PRODUCT && method != QT_GRID_KMEANS)
        return fail(ctx, QT_EINVAL, "unknown grid method %d", method);
    if (tol <= 0) tol = 1e-14;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    std::map<long long, std::vector<double>> base;   // N -> base grid of N(0, I_d), [N][d]
    for (int k = 0; k <= n; ++k) {
        const long long Nk = model->N[k];
        if (base.count(Nk)) continue;
        std::vector<double> G((size_t)Nk * d, 0.0);
        if (Nk == 1) {
            // the single point is the mean
        } else if (method == QT_GRID_LLOYD1D) {
            std::vector<double> x = lloyd1d((int)Nk, tol);
            for (long long j = 0; j < Nk; ++j) G[j] = x[j];
        } else if (method == QT_GRID_PRODUCT) {
            std::vector<int> best, cur;
            double score = 0;
            factor_sizes((int)Nk, d, best, cur, score);
            std::sort(best.begin(), best.end());
            std::vector<std::vector<double>> ax;
            for (int l = 0; l < d; ++l) ax.push_back(lloyd1d(best[l], tol));
            for (long long j = 0; j < Nk; ++j) {
                long long r = j;
                for (int l = d - 1; l >= 0; --l) {
                    G[j * d + l] = ax[l][r % best[l]];
                    r /= best[l];
                }
            }
        } else {
            const long long S = samples > 0 ? samples : std::max<long long>(20 * Nk, 100000);
            const int its = iters > 0 ? iters : 20;
            if (S < Nk) return fail(ctx, QT_EINVAL, "k-means needs at least N training samples");
            void *dZ, *dC, *dsum, *dcnt;
            if ((s = dev_get(ctx, "km_Z", sizeof(float) * (size_t)S * d, &dZ))) return s;
            if ((s = dev_get(ctx, "km_C", sizeof(float) * (size_t)Nk * d, &dC))) return s;
            if ((s = dev_get(ctx, "km_sum", 8 * (size_t)Nk * d, &dsum))) return s;
            if ((s = dev_get(ctx, "km_cnt", 8 * (size_t)Nk, &dcnt))) return s;
            const unsigned long long kseed = seed ^ (0x9E3779B97F4A7C15ull * (unsigned long long)Nk);
            kmeans_draw_kernel<<<(unsigned)((S + 255) / 256), 256, 0, st>>>(d, kseed, S, (float*)dZ);
            QT_CUDA(cudaGetLastError());
            QT_CUDA(cudaMemcpyAsync(dC, dZ, sizeof(float) * (size_t)Nk * d, cudaMemcpyDeviceToDevice, st));
            const size_t csm = sizeof(float) * (size_t)Nk * d;
            const int use_smem = csm <= 160 * 1024;
            if (use_smem)
                QT_CUDA(cudaFuncSetAttribute(kmeans_assign_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)csm));
            for (int it = 0; it < its; ++it) {
                QT_CUDA(cudaMemsetAsync(dsum, 0, 8 * (size_t)Nk * d, st));
                QT_CUDA(cudaMemsetAsync(dcnt, 0, 8 * (size_t)Nk, st));
                kmeans_assign_kernel<<<(unsigned)((S + 255) / 256), 256, use_smem ? csm : 0, st>>>(
                    d, S, (const float*)dZ, (int)Nk, (const float*)dC, (unsigned long long*)dsum,
                    (unsigned long long*)dcnt, use_smem);
                QT_CUDA(cudaGetLastError());
                kmeans_update_kernel<<<(unsigned)((Nk + 255) / 256), 256, 0, st>>>(
                    d, (int)Nk, (const unsigned long long*)dsum, (const unsigned long long*)dcnt, (float*)dC);
                QT_CUDA(cudaGetLastError());
            }
            std::vector<float> Gf((size_t)Nk * d);
            QT_CUDA(cudaMemcpyAsync(Gf.data(), dC, csm, cudaMemcpyDeviceToHost, st));
            QT_CUDA(cudaStreamSynchronize(st));
            for (size_t e = 0; e < Gf.size(); ++e) G[e] = (double)Gf[e];
        }
        base[Nk] = std::move(G);
    }
    // map every layer: x = m_k + L_k g
    long long off = 0;
    void *dG, *dm, *dL;
    long long maxN = 0;
    for (int k = 0; k <= n; ++k) maxN = std::max<long long>(maxN, model->N[k]);
    if ((s = dev_get(ctx, "bg_G", sizeof(double) * (size_t)maxN * d, &dG))) return s;
    if ((s = dev_get(ctx, "bg_m", sizeof(double) * d, &dm))) return s;
    if ((s = dev_get(ctx, "bg_L", sizeof(double) * d * d, &dL))) return s;
    for (int k = 0; k <= n; ++k) {
        const long long Nk = model->N[k];
        const std::vector<double>& G = base[Nk];
        QT_CUDA(cudaMemcpyAsync(dG, G.data(), sizeof(double) * (size_t)Nk * d, cudaMemcpyHostToDevice, st));
        QT_CUDA(cudaMemcpyAsync(dm, model->m + (long long)k * d, sizeof(double) * d, cudaMemcpyHostToDevice, st));
        QT_CUDA(cudaMemcpyAsync(dL, model->L + (long long)k * d * d, sizeof(double) * d * d, cudaMemcpyHostToDevice, st));
        map_grid_kernel<<<(unsigned)((Nk + 255) / 256), 256, 0, st>>>(d, (int)Nk, (const double*)dG,
                                                                    (const double*)dm, (const double*)dL,
                                                                    grids + off * d);
        QT_CUDA(cudaGetLastError());
        QT_CUDA(cudaStreamSynchronize(st));  // the staging buffers are reused next layer
        off += Nk;
    }
    return QT_OK;
}
