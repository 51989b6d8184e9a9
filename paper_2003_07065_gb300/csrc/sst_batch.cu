// Batched execution of many channels (plans) of uneven lengths and mixed
// (hop, nfft, band, z): persistent CTAs walk device tables of work items, one
// launch per (kernel, nfft) group, the groups of a phase on parallel streams,
// optionally captured once into a CUDA graph and replayed.  An autotuner
// times candidate work granularities and grid sizes on the real batch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "sst_internal.h"
#include "sst_kernels.cuh"

namespace sst {

// one CTA per channel: reduce the channel's pre-pass partials into its scalars
// (same arithmetic as k_gamma)
__global__ void k_gamma_batch(BatchChan *__restrict__ ch, int nchan, const float *__restrict__ partial) {
    __shared__ float red[32];
    const int c = blockIdx.x;
    if (c >= nchan) return;
    const BatchChan &b = ch[c];
    float v = 0.f;
    for (int i = threadIdx.x; i < b.nparts; i += blockDim.x) v = fmaxf(v, partial[b.part0 + i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float r = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, red[w]);
        *b.sc = scalars_from_max(r, b.frac2, b.d.relative ? 0 : 1, b.sum_abs_g, b.d.log2_nb);
    }
}

__global__ void k_finalize_batch(const BatchChan *__restrict__ ch, const BatchItem *__restrict__ items, int nitems) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem w = items[it];
        const BatchChan &c = ch[w.chan];
        for (int64_t p = w.begin + threadIdx.x; p < w.end; p += blockDim.x)
            c.xhat[p - c.poff] = finalize_value(c.d, c.ola, p);
    }
}

}  // namespace sst

using namespace sst;

namespace {

struct Knobs {
    int fwd_frames = 16;   // frames per forward work item
    int abs_quads = 8;     // frame quads per pre-pass work item
    int grid_mul = 1;      // persistent CTAs per SM = occupancy x grid_mul
};
constexpr int kMinAbsQuads = 2;   // finest pre-pass granularity the tuner tries

struct Group {
    int kind;              // KIND_B_*
    int nf;
    const KernelTable *kt;
    std::vector<BatchItem> items;
    BatchItem *d_items = nullptr;
    int grid = 0;
    size_t smem = 0;
    int max_nbo = 0;
    int part_off = 0;      // pre-pass groups: first partial slot
};

std::mutex g_tune_mu;
std::map<std::string, Knobs> g_tune_cache;

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

struct sst_batch {
    int device = 0;
    int nsm = 0;
    uint32_t flags = 0;
    std::vector<sst_batch_item> items;
    std::vector<BatchChan> ch;
    BatchChan *d_ch = nullptr;
    std::vector<Group> groups;   // pre-pass groups, then forward, then inverse
    std::vector<BatchItem> fin;
    BatchItem *d_fin = nullptr;
    int total_parts = 0;
    size_t ws_bytes = 0;
    std::vector<size_t> off_sc, off_ola;
    size_t off_part = 0;
    void *bound_ws = nullptr;
    std::vector<cudaStream_t> side;  // fork streams
    cudaStream_t cap = nullptr;      // capture stream (the caller's may be the legacy stream)
    std::vector<cudaEvent_t> ev;     // fork / join events
    cudaGraphExec_t gexec = nullptr;
    void *graph_ws = nullptr;
    int graph_kernels = 0;           // kernels per graph replay
    Knobs knobs;
    std::string signature;
};

namespace {

void free_items(sst_batch *b) {
    for (auto &g : b->groups)
        if (g.d_items) cudaFree(g.d_items);
    b->groups.clear();
    if (b->d_fin) cudaFree(b->d_fin);
    b->d_fin = nullptr;
}

void drop_graph(sst_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->graph_ws = nullptr;
}

// work items and launch shapes for the current knobs
sst_status build_items(sst_batch *b) {
    free_items(b);
    drop_graph(b);
    const int nch = (int)b->ch.size();
    std::map<int, std::vector<int>> by_nf;
    for (int c = 0; c < nch; ++c) by_nf[b->ch[c].d.nf].push_back(c);
    // pre-pass groups; a channel's partials are contiguous
    int part = 0;
    for (auto &kv : by_nf) {
        Group g;
        g.kind = KIND_B_ABSMAX;
        g.nf = kv.first;
        g.kt = table_for_nf(kv.first);
        g.part_off = part;
        for (int c : kv.second) {
            const SstDev &d = b->ch[c].d;
            b->ch[c].part0 = part;
            const int64_t units = d.relative ? (d.F + 3) / 4 : d.n;
            const int64_t step = d.relative ? b->knobs.abs_quads : (int64_t)b->knobs.abs_quads * 4 * d.hop * 64;
            int cnt = 0;
            for (int64_t u = 0; u < units; u += step, ++cnt) g.items.push_back({c, 0, u, std::min(units, u + step)});
            b->ch[c].nparts = cnt;
            part += cnt;
        }
        g.smem = 2 * g.kt->smem_frame;
        b->groups.push_back(std::move(g));
    }
    b->total_parts = part;
    // forward and inverse groups by (nf, pruning class): a channel with a
    // half-length window and a band of class 1 or 2 runs the pruned kernels
    auto class_of = [](const SstDev &d, const KernelTable *kt) {
        return d.L <= d.nf / 2 + 1 ? band_class(d.nf, kt->r1, d.k_hi) : 0;
    };
    std::map<std::pair<int, int>, std::vector<int>> by_fwd;
    for (int c = 0; c < nch; ++c) {
        const SstDev &d = b->ch[c].d;
        by_fwd[{d.nf, class_of(d, table_for_nf(d.nf))}].push_back(c);
    }
    for (auto &kv : by_fwd) {
        Group g;
        const int cls = kv.first.second;
        g.kind = kind_cls(KIND_B_FWD, cls);
        g.nf = kv.first.first;
        g.kt = table_for_nf(g.nf);
        // interleave the channels' chunks so long channels do not end last
        std::vector<std::vector<BatchItem>> per;
        for (int c : kv.second) {
            const SstDev &d = b->ch[c].d;
            std::vector<BatchItem> v;
            for (int64_t m = 0; m < d.F; m += b->knobs.fwd_frames) v.push_back({c, 0, m, std::min(d.F, m + b->knobs.fwd_frames)});
            per.push_back(std::move(v));
            g.max_nbo = std::max(g.max_nbo, d.nbo);
        }
        for (size_t r = 0;; ++r) {
            bool any = false;
            for (auto &v : per)
                if (r < v.size()) { g.items.push_back(v[r]); any = true; }
            if (!any) break;
        }
        g.smem = g.kt->smem_frame + tacc_bytes(g.max_nbo) + (cls > 0 ? mirror_bytes(g.max_nbo) : 0);
        b->groups.push_back(std::move(g));
    }
    // inverse groups, by (nf, window and pruning class)
    std::map<std::pair<int, int>, std::vector<int>> by_inv;
    for (int c = 0; c < nch; ++c) {
        const SstDev &d = b->ch[c].d;
        by_inv[{d.nf, d.L <= d.nf / 2 + 1 ? kind_cls(KIND_B_INV, class_of(d, table_for_nf(d.nf)))
                      : d.L > d.nf + 1    ? KIND_B_INV_LONG
                                          : KIND_B_INV_WIDE}].push_back(c);
    }
    for (auto &kv : by_inv) {
        Group g;
        g.kind = kv.first.second;
        g.nf = kv.first.first;
        g.kt = table_for_nf(g.nf);
        std::vector<std::vector<BatchItem>> per;
        for (int c : kv.second) {
            const SstDev &d = b->ch[c].d;
            std::vector<BatchItem> v;
            for (int64_t t = 0; t < d.ntiles; ++t) v.push_back({c, 0, t, t + 1});
            per.push_back(std::move(v));
            g.smem = std::max(g.smem, inverse_smem_bytes(g.kt->smem_frame, d.z, d.k_hi - d.k_lo + 1, d.seg_len));
        }
        for (size_t r = 0;; ++r) {
            bool any = false;
            for (auto &v : per)
                if (r < v.size()) { g.items.push_back(v[r]); any = true; }
            if (!any) break;
        }
        b->groups.push_back(std::move(g));
    }
    // finalize items
    b->fin.clear();
    for (int c = 0; c < nch; ++c)
        for (int64_t p = 0; p < b->ch[c].d.n; p += 65536) b->fin.push_back({c, 0, p, std::min(b->ch[c].d.n, p + 65536)});
    // shapes, uploads
    for (auto &g : b->groups) {
        cudaError_t e = raise_smem(g.kt, g.kind, g.smem);
        if (e != cudaSuccess) return cuda_fail(e, "batch cudaFuncSetAttribute");
        int occ = 1;
        if (g.kt->occupancy(g.kind, g.smem, &occ) != cudaSuccess || occ < 1) occ = 1;
        g.grid = (int)std::min<int64_t>((int64_t)occ * b->nsm * b->knobs.grid_mul, (int64_t)g.items.size());
        if (g.grid < 1) g.grid = 1;
        const size_t bytes = sizeof(BatchItem) * std::max<size_t>(g.items.size(), 1);
        if (cudaMalloc(&g.d_items, bytes) != cudaSuccess) return fail(SST_ENOMEM, "batch item table");
        e = cudaMemcpy(g.d_items, g.items.data(), sizeof(BatchItem) * g.items.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "batch item upload");
    }
    if (cudaMalloc(&b->d_fin, sizeof(BatchItem) * std::max<size_t>(b->fin.size(), 1)) != cudaSuccess)
        return fail(SST_ENOMEM, "batch item table");
    cudaError_t e = cudaMemcpy(b->d_fin, b->fin.data(), sizeof(BatchItem) * b->fin.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "batch item upload");
    // workspace layout: per channel scalars and overlap-add partials, then the pre-pass partials
    size_t off = 0;
    b->off_sc.assign(nch, 0);
    b->off_ola.assign(nch, 0);
    for (int c = 0; c < nch; ++c) {
        b->off_sc[c] = off;
        off = align256(off + sizeof(SstScalars));
        b->off_ola[c] = off;
        off = align256(off + sizeof(float) * (size_t)b->ch[c].d.ntiles * b->ch[c].d.seg_len);
    }
    b->off_part = off;
    // size the pre-pass partials for the finest granularity the tuner tries
    // (kMinAbsQuads), so a workspace sized at creation fits every knob setting
    int64_t max_parts = 0;
    for (int c = 0; c < nch; ++c) {
        const SstDev &d = b->ch[c].d;
        const int64_t units = d.relative ? (d.F + 3) / 4 : d.n;
        const int64_t step = d.relative ? kMinAbsQuads : (int64_t)kMinAbsQuads * 4 * d.hop * 64;
        max_parts += (units + step - 1) / step;
    }
    max_parts = std::max<int64_t>(max_parts, b->total_parts);
    b->ws_bytes = align256(off + sizeof(float) * (size_t)std::max<int64_t>(max_parts, 1));
    b->bound_ws = nullptr;
    return SST_OK;
}

// point the channel table at workspace ws (re-uploads the table)
sst_status bind(sst_batch *b, void *ws, cudaStream_t st) {
    if (b->bound_ws == ws) return SST_OK;
    char *base = (char *)ws;
    for (size_t c = 0; c < b->ch.size(); ++c) {
        b->ch[c].sc = (SstScalars *)(base + b->off_sc[c]);
        b->ch[c].ola = (float *)(base + b->off_ola[c]);
    }
    SST_CU(cudaMemcpyAsync(b->d_ch, b->ch.data(), sizeof(BatchChan) * b->ch.size(), cudaMemcpyHostToDevice, st),
           "batch channel table upload");
    SST_CU(cudaStreamSynchronize(st), "batch channel table upload");
    b->bound_ws = ws;
    drop_graph(b);
    return SST_OK;
}

// Enqueue one phase: the groups of `kind` (a predicate) on forked streams.
template <class Pred>
sst_status enqueue_phase(sst_batch *b, cudaStream_t st, float *part, bool count, Pred pred) {
    std::vector<Group *> gs;
    for (auto &g : b->groups)
        if (pred(g.kind)) gs.push_back(&g);
    if (gs.empty()) return SST_OK;
    // fork: side streams wait for the main stream (more groups than streams
    // share them round-robin)
    const size_t nstreams = std::min(gs.size(), b->side.size() + 1);
    SST_CU(cudaEventRecord(b->ev[0], st), "batch fork");
    for (size_t i = 1; i < nstreams; ++i) SST_CU(cudaStreamWaitEvent(b->side[i - 1], b->ev[0], 0), "batch fork");
    for (size_t i = 0; i < gs.size(); ++i) {
        Group &g = *gs[i];
        const size_t k = i % nstreams;
        cudaStream_t s = k == 0 ? st : b->side[k - 1];
        cudaError_t e = g.kt->batch(g.kind, b->d_ch, g.d_items, (int)g.items.size(), g.max_nbo, g.grid, g.smem,
                                    part + g.part_off, s);
        if (e != cudaSuccess) return cuda_fail(e, "batch launch");
        if (count) count_launch();
    }
    // join
    for (size_t i = 1; i < nstreams; ++i) {
        SST_CU(cudaEventRecord(b->ev[i], b->side[i - 1]), "batch join");
        SST_CU(cudaStreamWaitEvent(st, b->ev[i], 0), "batch join");
    }
    return SST_OK;
}

// count = false while capturing a graph: the replays are counted instead
sst_status enqueue_all(sst_batch *b, void *ws, cudaStream_t st, bool count) {
    float *part = (float *)((char *)ws + b->off_part);
    sst_status s = enqueue_phase(b, st, part, count, [](int k) { return k == KIND_B_ABSMAX; });
    if (s != SST_OK) return s;
    k_gamma_batch<<<(unsigned)b->ch.size(), 256, 0, st>>>(b->d_ch, (int)b->ch.size(), part);
    SST_CU(cudaGetLastError(), "batch gamma launch");
    if (count) count_launch();
    s = enqueue_phase(b, st, part, count, [](int k) { return (k & ((1 << KIND_CLS_SHIFT) - 1)) == KIND_B_FWD; });
    if (s != SST_OK) return s;
    s = enqueue_phase(b, st, part, count, [](int k) {
        const int base = k & ((1 << KIND_CLS_SHIFT) - 1);
        return base == KIND_B_INV || base == KIND_B_INV_WIDE || base == KIND_B_INV_LONG;
    });
    if (s != SST_OK) return s;
    const int grid = (int)std::min<size_t>(std::max<size_t>(b->fin.size(), 1), (size_t)b->nsm * 8);
    k_finalize_batch<<<grid, 256, 0, st>>>(b->d_ch, b->d_fin, (int)b->fin.size());
    SST_CU(cudaGetLastError(), "batch finalize launch");
    if (count) count_launch();
    return SST_OK;
}

sst_status run(sst_batch *b, void *ws, cudaStream_t st) {
    sst_status s = bind(b, ws, st);
    if (s != SST_OK) return s;
    if (!(b->flags & SST_BATCH_GRAPH)) return enqueue_all(b, ws, st, true);
    if (!b->gexec || b->graph_ws != ws) {
        drop_graph(b);
        // capture on the batch's own stream; the graph is launched on the caller's
        SST_CU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "graph capture begin");
        s = enqueue_all(b, ws, b->cap, false);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
        if (s != SST_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return cuda_fail(e, "graph capture end");
        e = cudaGraphInstantiate(&b->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->gexec = nullptr;
            return cuda_fail(e, "graph instantiate");
        }
        b->graph_ws = ws;
        b->graph_kernels = 0;
        for (auto &g : b->groups) b->graph_kernels += 1;
        b->graph_kernels += 2;   // per-channel thresholds and finalize
    }
    SST_CU(cudaGraphLaunch(b->gexec, st), "graph launch");
    for (int k = 0; k < b->graph_kernels; ++k) count_launch();
    return SST_OK;
}

std::string gpu_name(int dev) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    return p.name;
}

std::string make_signature(const sst_batch *b) {
    // the batch's shape class: sorted (nf, L, hop, band bins, z, relative, log2 n) tuples + the GPU
    std::vector<std::string> parts;
    for (auto &c : b->ch) {
        char s[160];
        snprintf(s, sizeof s, "%d/%d/%d/%d/%d/%d/%d", c.d.nf, c.d.L, c.d.hop, c.d.nb, c.d.z, c.d.relative,
                 (int)std::log2((double)std::max<int64_t>(c.d.n, 1)));
        parts.push_back(s);
    }
    std::sort(parts.begin(), parts.end());
    std::string sig = gpu_name(b->device);
    for (auto &p : parts) sig += ";" + p;
    return sig;
}

void cache_load_file() {
    const char *path = getenv("SST_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[1 << 16];
    while (fgets(line, sizeof line, f)) {
        char *tab = strrchr(line, '\t');
        if (!tab) continue;
        *tab = 0;
        Knobs k;
        if (sscanf(tab + 1, "%d %d %d", &k.fwd_frames, &k.abs_quads, &k.grid_mul) == 3) g_tune_cache[line] = k;
    }
    fclose(f);
}

void cache_store_file(const std::string &sig, const Knobs &k) {
    const char *path = getenv("SST_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s\t%d %d %d\n", sig.c_str(), k.fwd_frames, k.abs_quads, k.grid_mul);
    fclose(f);
}

}  // namespace

SST_API sst_status sst_batch_create(const sst_batch_item *items, int32_t count, uint32_t flags, sst_batch_t *out) {
    SST_NVTX_RANGE();
    if (!out) return fail(SST_EINVAL, "out is NULL");
    *out = nullptr;
    if (!items || count < 1) return fail(SST_EINVAL, "need at least one batch item");
    if (flags & ~(SST_BATCH_GRAPH)) return fail(SST_EINVAL, "unknown batch flags 0x%x", flags);
    int dev = -1;
    SST_CU(cudaGetDevice(&dev), "cudaGetDevice");
    for (int i = 0; i < count; ++i) {
        const sst_batch_item &it = items[i];
        if (!it.plan) return fail(SST_EINVAL, "item %d: plan is NULL", i);
        if (it.plan->device != dev) return fail(SST_EINVAL, "item %d: plan is on device %d, current is %d", i, it.plan->device, dev);
        if (it.n != it.plan->d.n) return fail(SST_EINVAL, "item %d: n = %lld differs from its plan's n", i, (long long)it.n);
        if (!it.x || !it.tfr || !it.xhat) return fail(SST_EINVAL, "item %d: NULL buffer", i);
    }
    sst_batch *b = new (std::nothrow) sst_batch();
    if (!b) return fail(SST_ENOMEM, "host allocation failed");
    b->device = dev;
    b->flags = flags;
    b->items.assign(items, items + count);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) { delete b; return fail(SST_ECUDA, "device query"); }
    b->nsm = prop.multiProcessorCount;
    b->ch.resize(count);
    for (int i = 0; i < count; ++i) {
        BatchChan &c = b->ch[i];
        memset(&c, 0, sizeof c);
        c.d = items[i].plan->d;
        c.x = items[i].x;
        c.T = (float2 *)items[i].tfr;
        c.xhat = items[i].xhat;
        c.frac2 = items[i].plan->gamma_frac2;
        c.sum_abs_g = items[i].plan->sum_abs_g;
    }
    if (cudaMalloc(&b->d_ch, sizeof(BatchChan) * count) != cudaSuccess) { delete b; return fail(SST_ENOMEM, "batch channel table"); }
    b->side.resize(16, nullptr);
    b->ev.resize(17, nullptr);
    for (auto &s : b->side) cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    for (auto &e : b->ev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    b->signature = make_signature(b);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (g_tune_cache.empty()) cache_load_file();
        auto it = g_tune_cache.find(b->signature);
        if (it != g_tune_cache.end()) b->knobs = it->second;
    }
    sst_status s = build_items(b);
    if (s != SST_OK) { sst_batch_destroy(b); return s; }
    *out = b;
    return SST_OK;
}

SST_API sst_status sst_batch_workspace(sst_batch_t b, size_t *bytes) {
    if (!b || !bytes) return fail(SST_EINVAL, "NULL argument");
    *bytes = b->ws_bytes;
    return SST_OK;
}

SST_API sst_status sst_batch_run(sst_batch_t b, void *ws, void *stream) {
    SST_NVTX_RANGE();
    if (!b) return fail(SST_EINVAL, "batch is NULL");
    if (!ws || (((uintptr_t)ws) & 255)) return fail(SST_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    int dev = -1;
    SST_CU(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != b->device) return fail(SST_EINVAL, "batch was created on device %d, current is %d", b->device, dev);
    return run(b, ws, (cudaStream_t)stream);
}

SST_API sst_status sst_batch_tune(sst_batch_t b, void *ws, void *stream, double *untuned_ms, double *tuned_ms) {
    SST_NVTX_RANGE();
    if (!b) return fail(SST_EINVAL, "batch is NULL");
    if (!ws || (((uintptr_t)ws) & 255)) return fail(SST_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t saved_flags = b->flags;
    b->flags &= ~SST_BATCH_GRAPH;   // time plain launches
    cudaEvent_t e0, e1;
    SST_CU(cudaEventCreate(&e0), "event");
    SST_CU(cudaEventCreate(&e1), "event");
    auto time_knobs = [&](const Knobs &k, double *ms) -> sst_status {
        b->knobs = k;
        sst_status s = build_items(b);
        if (s != SST_OK) return s;
        s = run(b, ws, st);  // warm-up (and rebinding)
        if (s != SST_OK) return s;
        SST_CU(cudaEventRecord(e0, st), "event");
        for (int r = 0; r < 3; ++r) {
            s = run(b, ws, st);
            if (s != SST_OK) return s;
        }
        SST_CU(cudaEventRecord(e1, st), "event");
        SST_CU(cudaEventSynchronize(e1), "event");
        float t = 0.f;
        SST_CU(cudaEventElapsedTime(&t, e0, e1), "event");
        *ms = t / 3.0;
        return SST_OK;
    };
    // candidate knobs; the first is the untuned default
    std::vector<Knobs> cands;
    const Knobs def;
    cands.push_back(def);
    for (int ff : {4, 16, 64})
        for (int aq : {kMinAbsQuads, 8, 32})
            for (int gm : {1, 2}) {
                Knobs k;
                k.fwd_frames = ff;
                k.abs_quads = aq;
                k.grid_mul = gm;
                if (k.fwd_frames == def.fwd_frames && k.abs_quads == def.abs_quads && k.grid_mul == def.grid_mul) continue;
                cands.push_back(k);
            }
    double best = 1e300, first = 0.0;
    Knobs bestk = def;
    sst_status s = SST_OK;
    for (size_t i = 0; i < cands.size() && s == SST_OK; ++i) {
        double ms = 0.0;
        s = time_knobs(cands[i], &ms);
        if (s != SST_OK) break;
        if (i == 0) first = ms;
        if (ms < best) { best = ms; bestk = cands[i]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->flags = saved_flags;
    if (s != SST_OK) return s;
    b->knobs = bestk;
    s = build_items(b);
    if (s != SST_OK) return s;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[b->signature] = bestk;
    }
    cache_store_file(b->signature, bestk);
    if (untuned_ms) *untuned_ms = first;
    if (tuned_ms) *tuned_ms = best;
    return SST_OK;
}

SST_API sst_status sst_batch_knobs(sst_batch_t b, int32_t *fwd_frames, int32_t *abs_quads, int32_t *grid_mul) {
    if (!b) return fail(SST_EINVAL, "batch is NULL");
    if (fwd_frames) *fwd_frames = b->knobs.fwd_frames;
    if (abs_quads) *abs_quads = b->knobs.abs_quads;
    if (grid_mul) *grid_mul = b->knobs.grid_mul;
    return SST_OK;
}

SST_API void sst_batch_destroy(sst_batch_t b) {
    if (!b) return;
    drop_graph(b);
    free_items(b);
    if (b->d_ch) cudaFree(b->d_ch);
    for (auto &s : b->side)
        if (s) cudaStreamDestroy(s);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (auto &e : b->ev)
        if (e) cudaEventDestroy(e);
    delete b;
}

SST_API sst_status sst_batch_submit(const sst_batch_item *items, int32_t count, void *ws, size_t ws_bytes,
                                    void *stream) {
    SST_NVTX_RANGE();
    sst_batch_t b = nullptr;
    sst_status s = sst_batch_create(items, count, 0, &b);
    if (s != SST_OK) return s;
    if (ws_bytes < b->ws_bytes) {
        const size_t need = b->ws_bytes;
        sst_batch_destroy(b);
        return fail(SST_EINVAL, "workspace of %zu bytes is smaller than the %zu bytes needed", ws_bytes, need);
    }
    s = sst_batch_run(b, ws, stream);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    sst_batch_destroy(b);
    if (s != SST_OK) return s;
    if (e != cudaSuccess) return cuda_fail(e, "batch synchronise");
    return SST_OK;
}

SST_API sst_status sst_batch_workspace_for(const sst_batch_item *items, int32_t count, size_t *bytes) {
    if (!bytes) return fail(SST_EINVAL, "bytes is NULL");
    sst_batch_t b = nullptr;
    sst_status s = sst_batch_create(items, count, 0, &b);
    if (s != SST_OK) return s;
    *bytes = b->ws_bytes;
    sst_batch_destroy(b);
    return SST_OK;
}
