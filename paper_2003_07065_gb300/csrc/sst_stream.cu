// Streaming service: many sensor streams push chunks; each tick batches the
// work every stream has ready (frames whose window has fully arrived, inverse
// tiles whose frames are all transformed, output samples no later frame
// touches) into shared launches of the batched kernels.  Per-stream state
// stays on the device: the signal tail, ring buffers of TFR rows and
// overlap-add tiles, and the cursors.  Tiles are cut from frame 0 with a fixed
// size, so a stream's results do not depend on how its data was chunked or
// mixed with other streams.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <vector>

#include "sst_internal.h"
#include "sst_kernels.cuh"

using namespace sst;

namespace {

constexpr int kStreamB = 16;          // frames per inverse tile of a stream
constexpr int kFwdFrames = 16;        // frames per forward work item

// the batched inverse kind for a stream's window (half length, up to nf + 1, longer)
int inv_kind_of(const SstDev &d) {
    return d.L <= d.nf / 2 + 1 ? KIND_B_INV : d.L > d.nf + 1 ? KIND_B_INV_LONG : KIND_B_INV_WIDE;
}

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Chunk {
    std::vector<float> data;
    double t_arrival;
};

struct Stream {
    bool used = false, closing = false, done = false;
    sst_plan_t plan = nullptr;
    SstDev base;                     // device view of the plan's tables, stream layout
    std::vector<double> g;           // FP64 window, for the edge normalisers at close
    float amp_bound = 0.f;
    int64_t max_chunk = 0;
    bool xhat_only = false;          // TFR columns are not copied to the host
    // device state (one allocation)
    void *dmem = nullptr;
    size_t dev_bytes = 0;
    float *sig = nullptr;
    int64_t sig_cap = 0, sig_base = 0, sig_end = 0;
    float2 *T = nullptr;
    int trow_cap = 0;
    float *ola = nullptr;
    int tile_cap = 0;
    float *xout = nullptr;
    int64_t xout_cap = 0;
    SstScalars *sc = nullptr;
    float *rd_left = nullptr, *rd_right = nullptr;   // edge normalisers written at close
    int64_t rd_cap = 0;
    // cursors (global frame / tile / sample indices)
    int64_t m_next = 0, t_next = 0, p_next = 0;
    int64_t N = -1;                  // total length once closed
    // host side
    std::deque<Chunk> pending;
    std::vector<float> tfr_host;     // finished rows, interleaved complex
    int64_t tfr_first = 0;           // frame of the first row in tfr_host
    std::vector<float> x_host;
    int64_t x_first = 0;
};

}  // namespace

struct sst_service {
    int device = 0;
    int nsm = 0;
    int max_streams = 0;
    size_t budget = 0, used = 0;
    std::vector<Stream> s;
    cudaStream_t st = nullptr;
    // pinned staging
    char *pin = nullptr;
    size_t pin_cap = 0;
    BatchChan *d_ch = nullptr;
    int d_ch_cap = 0;
    BatchItem *d_items = nullptr;
    int d_items_cap = 0;
    std::vector<double> lat;         // seconds, one per consumed chunk
    std::mutex mu;
};

namespace {

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

sst_status ensure_pinned(sst_service *sv, size_t bytes) {
    if (bytes <= sv->pin_cap) return SST_OK;
    if (sv->pin) cudaFreeHost(sv->pin);
    sv->pin = nullptr;
    size_t cap = std::max(bytes, sv->pin_cap * 2);
    if (cudaMallocHost(&sv->pin, cap) != cudaSuccess) {
        sv->pin_cap = 0;
        return fail(SST_ENOMEM, "pinned staging of %zu bytes", cap);
    }
    sv->pin_cap = cap;
    return SST_OK;
}

template <class T> sst_status ensure_dev(T **p, int *cap, int need) {
    if (need <= *cap) return SST_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    int c = std::max(need, *cap * 2);
    if (cudaMalloc(p, sizeof(T) * (size_t)c) != cudaSuccess) {
        *cap = 0;
        return fail(SST_ENOMEM, "service table");
    }
    *cap = c;
    return SST_OK;
}

// exact edge normalisers of a closed stream of N samples (Eq. 26, FP64)
void edge_tables(const Stream &S, int64_t N, std::vector<float> &left, std::vector<float> &right, int64_t &EL,
                 int64_t &ER) {
    const int M = S.base.M, hop = S.base.hop;
    const int64_t F = (N + hop - 1) / hop;
    auto D = [&](int64_t q) {
        int64_t mlo = (q - M > 0) ? (q - M + hop - 1) / hop : 0;
        int64_t mhi = (q + M) / hop;
        if (mhi > F - 1) mhi = F - 1;
        double s = 0.0;
        for (int64_t m = mlo; m <= mhi; ++m) {
            const int64_t j = q - m * hop;
            if (j >= -M && j <= M) s += S.g[j + M];
        }
        return S.g[M] * s;
    };
    EL = std::min<int64_t>(N, M);
    ER = std::max<int64_t>(EL, std::min<int64_t>(N, F * hop - M));
    left.resize(std::max<int64_t>(EL, 1));
    right.resize(std::max<int64_t>(N - ER, 1));
    for (int64_t q = 0; q < EL; ++q) left[q] = (float)(1.0 / D(q));
    for (int64_t q = ER; q < N; ++q) right[q - ER] = (float)(1.0 / D(q));
}

}  // namespace

SST_API sst_status sst_service_create(int32_t max_streams, size_t mem_budget, sst_service_t *out) {
    if (!out) return fail(SST_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_streams < 1 || max_streams > 4096) return fail(SST_EINVAL, "max_streams must be in [1, 4096]");
    int dev = -1;
    SST_CU(cudaGetDevice(&dev), "cudaGetDevice");
    sst_service *sv = new (std::nothrow) sst_service();
    if (!sv) return fail(SST_ENOMEM, "host allocation failed");
    sv->device = dev;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) { delete sv; return fail(SST_ECUDA, "device query"); }
    sv->nsm = prop.multiProcessorCount;
    sv->max_streams = max_streams;
    sv->budget = mem_budget;
    sv->s.resize(max_streams);
    if (cudaStreamCreateWithFlags(&sv->st, cudaStreamNonBlocking) != cudaSuccess) {
        delete sv;
        return fail(SST_ECUDA, "service stream");
    }
    *out = sv;
    return SST_OK;
}

SST_API sst_status sst_stream_open(sst_service_t sv, const sst_params *params, float amp_bound, int64_t max_chunk,
                                   int32_t *id) {
    SST_NVTX_RANGE();
    if (!sv || !params || !id) return fail(SST_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (params->flags & SST_GAMMA_RELATIVE)
        return fail(SST_EUNSUPPORTED, "streams need an absolute threshold (the whole-signal max is not known)");
    if (!(amp_bound > 0.f) || !std::isfinite(amp_bound)) return fail(SST_EINVAL, "amp_bound must be finite and > 0");
    if (max_chunk < 1) return fail(SST_EINVAL, "max_chunk must be >= 1");
    int slot = -1;
    for (int i = 0; i < sv->max_streams; ++i)
        if (!sv->s[i].used) { slot = i; break; }
    if (slot < 0) return fail(SST_EBUSY, "all %d stream slots are in use", sv->max_streams);
    // the plan supplies the tables; its own length only sizes its edge tables
    sst_params p = *params;
    p.n = 4 * (int64_t)p.L;
    const bool xhat_only = (p.flags & SST_STREAM_XHAT_ONLY) != 0;
    p.flags &= ~SST_STREAM_XHAT_ONLY;
    sst_plan_t plan = nullptr;
    sst_status st = sst_plan_create(&p, &plan);
    if (st != SST_OK) return st;
    Stream S;
    S.plan = plan;
    S.base = plan->d;
    S.amp_bound = amp_bound;
    S.max_chunk = max_chunk;
    S.xhat_only = xhat_only;
    SstDev &d = S.base;
    const int M = d.M, H = d.hop;
    // sizes: signal tail + a burst of pending data, twice over so compaction never overlaps
    const int64_t keep = (int64_t)d.L + (int64_t)kStreamB * H + 2 * H;
    const int64_t burst = 8 * max_chunk;
    S.sig_cap = 2 * (keep + burst);
    const int64_t frames_tick = burst / H + 2;
    S.trow_cap = (int)(frames_tick + 2 * kStreamB + 2);
    d.B = kStreamB;
    d.seg_len = (kStreamB - 1) * H + d.L;
    S.tile_cap = (int)(frames_tick / kStreamB + (d.L + (int64_t)kStreamB * H) / ((int64_t)kStreamB * H) + 4);
    S.xout_cap = burst + (int64_t)d.L + 2 * (int64_t)kStreamB * H;
    S.rd_cap = (int64_t)M + H + 1;
    size_t off = 0;
    const size_t o_sig = off; off = a256(off + sizeof(float) * S.sig_cap);
    const size_t o_T = off; off = a256(off + sizeof(float2) * (size_t)S.trow_cap * d.nbo);
    const size_t o_ola = off; off = a256(off + sizeof(float) * (size_t)S.tile_cap * d.seg_len);
    const size_t o_x = off; off = a256(off + sizeof(float) * S.xout_cap);
    const size_t o_sc = off; off = a256(off + sizeof(SstScalars));
    const size_t o_rl = off; off = a256(off + sizeof(float) * S.rd_cap);
    const size_t o_rr = off; off = a256(off + sizeof(float) * S.rd_cap);
    const size_t plan_bytes = 4096 + sizeof(float2) * (size_t)(2 * d.L + 2 * d.nf * (d.z + 1));
    S.dev_bytes = off + plan_bytes;
    if (sv->used + S.dev_bytes > sv->budget) {
        sst_plan_destroy(plan);
        return fail(SST_EBUSY, "stream needs %zu device bytes, %zu of the %zu-byte budget are left", S.dev_bytes,
                    sv->budget - sv->used, sv->budget);
    }
    if (cudaMalloc(&S.dmem, off) != cudaSuccess) {
        sst_plan_destroy(plan);
        return fail(SST_ENOMEM, "stream state of %zu bytes", off);
    }
    char *b = (char *)S.dmem;
    S.sig = (float *)(b + o_sig);
    S.T = (float2 *)(b + o_T);
    S.ola = (float *)(b + o_ola);
    S.xout = (float *)(b + o_x);
    S.sc = (SstScalars *)(b + o_sc);
    S.rd_left = (float *)(b + o_rl);
    S.rd_right = (float *)(b + o_rr);
    d.trow_cap = S.trow_cap;
    d.tile_cap = S.tile_cap;
    d.ER = INT64_MAX;                // no right edge until the stream closes
    // FP64 window for the edge normalisers
    S.g.resize(d.L);
    if (params->g) {
        for (int i = 0; i < d.L; ++i) S.g[i] = params->g[i];
    } else {
        const double amp = std::pow(M_PI * params->sigma * params->sigma, -0.25);
        for (int j = -M; j <= M; ++j) S.g[j + M] = amp * std::exp(-(double)j * j / (2.0 * params->sigma * params->sigma));
    }
    // fixed-point scale from the declared amplitude bound (as for absolute plans)
    SstScalars sc;
    memset(&sc, 0, sizeof sc);
    const float bound = amp_bound * plan->sum_abs_g;
    int e = 0;
    if (bound > 0.f && bound < 3.0e38f) {
        int ex;
        std::frexp(bound, &ex);
        e = SST_T_BITS - ex - d.log2_nb;
    }
    const int e1 = e / 2, e2 = e - e / 2;
    sc.s1 = std::ldexp(1.f, e1);
    sc.s2 = std::ldexp(1.f, e2);
    sc.r1 = std::ldexp(1.f, -e1);
    sc.r2 = std::ldexp(1.f, -e2);
    cudaError_t ce = cudaMemcpy(S.sc, &sc, sizeof sc, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        cudaFree(S.dmem);
        sst_plan_destroy(plan);
        return cuda_fail(ce, "stream scalars");
    }
    // kernel attributes for this stream's shapes
    const size_t smem_f = plan->kt->smem_frame + tacc_bytes(d.nbo);
    const size_t smem_i = inverse_smem_bytes(plan->kt->smem_frame, d.z, d.k_hi - d.k_lo + 1, d.seg_len);
    const int ik = inv_kind_of(d);
    if (raise_smem(plan->kt, KIND_B_FWD, smem_f) != cudaSuccess || raise_smem(plan->kt, ik, smem_i) != cudaSuccess) {
        cudaFree(S.dmem);
        sst_plan_destroy(plan);
        return fail(SST_EUNSUPPORTED, "stream kernel shared memory");
    }
    S.used = true;
    sv->used += S.dev_bytes;
    sv->s[slot] = std::move(S);
    *id = slot;
    return SST_OK;
}

SST_API sst_status sst_stream_push(sst_service_t sv, int32_t id, const float *chunk, int64_t n, double t_arrival) {
    if (!sv || !chunk) return fail(SST_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (id < 0 || id >= sv->max_streams || !sv->s[id].used) return fail(SST_EINVAL, "no open stream %d", id);
    Stream &S = sv->s[id];
    if (S.closing) return fail(SST_EINVAL, "stream %d is closed", id);
    if (n < 1 || n > S.max_chunk) return fail(SST_EINVAL, "chunk of %lld samples (max %lld)", (long long)n, (long long)S.max_chunk);
    int64_t queued = 0;
    for (auto &c : S.pending) queued += (int64_t)c.data.size();
    if (queued + n > 8 * S.max_chunk) return fail(SST_EBUSY, "stream %d has %lld samples queued", id, (long long)queued);
    Chunk c;
    c.data.assign(chunk, chunk + n);
    c.t_arrival = t_arrival >= 0.0 ? t_arrival : now_s();
    S.pending.push_back(std::move(c));
    return SST_OK;
}

SST_API sst_status sst_stream_close(sst_service_t sv, int32_t id) {
    if (!sv) return fail(SST_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (id < 0 || id >= sv->max_streams || !sv->s[id].used) return fail(SST_EINVAL, "no open stream %d", id);
    sv->s[id].closing = true;
    return SST_OK;
}

SST_API sst_status sst_service_tick(sst_service_t sv) {
    SST_NVTX_RANGE();
    if (!sv) return fail(SST_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    int dev = -1;
    SST_CU(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != sv->device) return fail(SST_EINVAL, "service was created on device %d, current is %d", sv->device, dev);
    cudaStream_t st = sv->st;
    struct Work {
        int id;
        int64_t m_ready, t_ready, p_ready;
        std::vector<double> arrivals;
    };
    std::vector<Work> work;
    // 1. bring pending chunks onto the device
    size_t pin_need = 0;
    for (auto &S : sv->s)
        if (S.used && !S.done)
            for (auto &c : S.pending) pin_need += sizeof(float) * c.data.size();
    sst_status s = ensure_pinned(sv, pin_need + 4096);
    if (s != SST_OK) return s;
    size_t pin_off = 0;
    for (int id = 0; id < sv->max_streams; ++id) {
        Stream &S = sv->s[id];
        if (!S.used || S.done) continue;
        Work w;
        w.id = id;
        const SstDev &d = S.base;
        if (!S.pending.empty()) {
            int64_t total = 0;
            for (auto &c : S.pending) total += (int64_t)c.data.size();
            // compact: keep from the first sample the next frame needs
            const int64_t keep_from = std::max<int64_t>(S.sig_base, S.m_next * d.hop - d.M);
            if ((S.sig_end - S.sig_base) + total > S.sig_cap) {
                const int64_t kept = S.sig_end - keep_from;
                if (kept + total > S.sig_cap) return fail(SST_EINTERNAL, "stream %d signal buffer overflow", id);
                if (kept > 0) {
                    // source and destination do not overlap: the buffer is twice the retained tail
                    SST_CU(cudaMemcpyAsync(S.sig, S.sig + (keep_from - S.sig_base), sizeof(float) * kept,
                                           cudaMemcpyDeviceToDevice, st), "signal compaction");
                }
                S.sig_base = keep_from;
            }
            for (auto &c : S.pending) {
                memcpy(sv->pin + pin_off, c.data.data(), sizeof(float) * c.data.size());
                SST_CU(cudaMemcpyAsync(S.sig + (S.sig_end - S.sig_base), sv->pin + pin_off, sizeof(float) * c.data.size(),
                                       cudaMemcpyHostToDevice, st), "chunk upload");
                pin_off += a256(sizeof(float) * c.data.size());
                S.sig_end += (int64_t)c.data.size();
                w.arrivals.push_back(c.t_arrival);
            }
            S.pending.clear();
        }
        // 2. what is ready
        const int H = d.hop, B = kStreamB;
        int64_t m_ready, t_ready, p_ready;
        if (S.closing) {
            const int64_t N = S.sig_end;
            const int64_t F = (N + H - 1) / H;
            m_ready = F;
            t_ready = (F + B - 1) / B;
            p_ready = N;
        } else {
            m_ready = (S.sig_end - 1 - d.M >= 0) ? (S.sig_end - 1 - d.M) / H + 1 : 0;
            t_ready = m_ready / B;
            p_ready = std::min<int64_t>(S.sig_end, std::max<int64_t>(S.p_next, t_ready * B * H - d.M));
        }
        // ring capacities bound the work of one tick
        m_ready = std::min<int64_t>(m_ready, S.t_next * B + S.trow_cap - B);
        if (!S.closing || m_ready < (S.sig_end + H - 1) / H) {
            t_ready = std::min<int64_t>(t_ready, m_ready / B);
            if (!S.closing) p_ready = std::min<int64_t>(p_ready, std::max<int64_t>(S.p_next, t_ready * B * H - d.M));
        }
        const int64_t first_live_tile = std::max<int64_t>(0, (S.p_next + d.M - d.seg_len + 1 + (int64_t)B * H - 1) / ((int64_t)B * H));
        t_ready = std::min<int64_t>(t_ready, first_live_tile + S.tile_cap);
        const bool all_tiles = S.closing && m_ready == (S.sig_end + H - 1) / H && t_ready == (m_ready + B - 1) / B;
        if (!all_tiles) p_ready = std::min<int64_t>(p_ready, std::max<int64_t>(S.p_next, t_ready * B * H - d.M));
        p_ready = std::min<int64_t>(p_ready, S.p_next + S.xout_cap);
        w.m_ready = m_ready;
        w.t_ready = t_ready;
        w.p_ready = p_ready;
        if (m_ready > S.m_next || t_ready > S.t_next || p_ready > S.p_next || !w.arrivals.empty()) work.push_back(std::move(w));
    }
    if (work.empty()) return SST_OK;
    // 3. channel table and items
    std::vector<BatchChan> ch(work.size());
    std::map<int, std::vector<BatchItem>> fwd, inv;   // by kernel-table key
    std::vector<BatchItem> fin;
    std::map<int, size_t> smem_f, smem_i;
    std::map<int, int> maxnbo;
    for (size_t i = 0; i < work.size(); ++i) {
        Stream &S = sv->s[work[i].id];
        BatchChan &c = ch[i];
        memset(&c, 0, sizeof c);
        c.d = S.base;
        const int64_t N = S.closing ? S.sig_end : -1;
        c.d.n = S.closing ? N : S.sig_end;
        c.d.F = S.closing ? (N + c.d.hop - 1) / c.d.hop : work[i].m_ready;
        c.d.ntiles = S.closing ? (c.d.F + kStreamB - 1) / kStreamB : work[i].t_ready;
        c.d.xoff = S.sig_base;
        if (S.closing) {
            std::vector<float> left, right;
            int64_t EL, ER;
            edge_tables(S, N, left, right, EL, ER);
            if ((int64_t)left.size() > S.rd_cap || (int64_t)right.size() > S.rd_cap)
                return fail(SST_EINTERNAL, "stream %d edge tables", work[i].id);
            SST_CU(cudaMemcpyAsync(S.rd_left, left.data(), sizeof(float) * left.size(), cudaMemcpyHostToDevice, st),
                   "edge tables");
            SST_CU(cudaMemcpyAsync(S.rd_right, right.data(), sizeof(float) * right.size(), cudaMemcpyHostToDevice, st),
                   "edge tables");
            SST_CU(cudaStreamSynchronize(st), "edge tables");   // the host vectors go out of scope
            c.d.EL = EL;
            c.d.ER = ER;
            c.d.rD_left = S.rd_left;
            c.d.rD_right = S.rd_right;
        }
        c.x = S.sig;
        c.T = S.T;
        c.xhat = S.xout;
        c.sc = S.sc;
        c.ola = S.ola;
        c.poff = S.p_next;
        const int nf = c.d.nf;
        const int ikey = nf * 32 + inv_kind_of(c.d);   // inverse group: (nf, kernel kind)
        for (int64_t m = S.m_next; m < work[i].m_ready; m += kFwdFrames)
            fwd[nf].push_back({(int)i, 0, m, std::min<int64_t>(work[i].m_ready, m + kFwdFrames)});
        for (int64_t t = S.t_next; t < work[i].t_ready; ++t) inv[ikey].push_back({(int)i, 0, t, t + 1});
        for (int64_t p = S.p_next; p < work[i].p_ready; p += 65536)
            fin.push_back({(int)i, 0, p, std::min<int64_t>(work[i].p_ready, p + 65536)});
        smem_f[nf] = std::max(smem_f[nf], S.plan->kt->smem_frame + tacc_bytes(c.d.nbo));
        maxnbo[nf] = std::max(maxnbo[nf], c.d.nbo);
        smem_i[ikey] = std::max(smem_i[ikey], inverse_smem_bytes(S.plan->kt->smem_frame, c.d.z, c.d.k_hi - c.d.k_lo + 1,
                                                                  c.d.seg_len));
    }
    std::vector<BatchItem> all;
    std::vector<std::pair<size_t, size_t>> spans_f, spans_i;
    std::vector<int> keys_f, keys_i;
    for (auto &kv : fwd) { spans_f.push_back({all.size(), kv.second.size()}); keys_f.push_back(kv.first); all.insert(all.end(), kv.second.begin(), kv.second.end()); }
    for (auto &kv : inv) { spans_i.push_back({all.size(), kv.second.size()}); keys_i.push_back(kv.first); all.insert(all.end(), kv.second.begin(), kv.second.end()); }
    const size_t fin_off = all.size();
    all.insert(all.end(), fin.begin(), fin.end());
    s = ensure_dev(&sv->d_ch, &sv->d_ch_cap, (int)ch.size());
    if (s != SST_OK) return s;
    s = ensure_dev(&sv->d_items, &sv->d_items_cap, (int)std::max<size_t>(all.size(), 1));
    if (s != SST_OK) return s;
    // tables go through pinned staging (after the chunk data)
    const size_t tb = a256(sizeof(BatchChan) * ch.size()) + a256(sizeof(BatchItem) * all.size());
    if (pin_off + tb > sv->pin_cap) {
        SST_CU(cudaStreamSynchronize(st), "staging");
        s = ensure_pinned(sv, pin_off + tb);
        if (s != SST_OK) return s;
    }
    memcpy(sv->pin + pin_off, ch.data(), sizeof(BatchChan) * ch.size());
    SST_CU(cudaMemcpyAsync(sv->d_ch, sv->pin + pin_off, sizeof(BatchChan) * ch.size(), cudaMemcpyHostToDevice, st), "tables");
    pin_off += a256(sizeof(BatchChan) * ch.size());
    if (!all.empty()) {
        memcpy(sv->pin + pin_off, all.data(), sizeof(BatchItem) * all.size());
        SST_CU(cudaMemcpyAsync(sv->d_items, sv->pin + pin_off, sizeof(BatchItem) * all.size(), cudaMemcpyHostToDevice, st),
               "tables");
    }
    // 4. launches: forward groups, inverse groups, finalize
    for (size_t g = 0; g < keys_f.size(); ++g) {
        const int nf = keys_f[g];
        const KernelTable *kt = table_for_nf(nf);
        int occ = 1;
        if (kt->occupancy(KIND_B_FWD, smem_f[nf], &occ) != cudaSuccess || occ < 1) occ = 1;
        const int grid = (int)std::min<int64_t>((int64_t)occ * sv->nsm, (int64_t)spans_f[g].second);
        cudaError_t e = kt->batch(KIND_B_FWD, sv->d_ch, sv->d_items + spans_f[g].first, (int)spans_f[g].second,
                                  maxnbo[nf], grid, smem_f[nf], nullptr, st);
        if (e != cudaSuccess) return cuda_fail(e, "stream forward launch");
        count_launch();
    }
    for (size_t g = 0; g < keys_i.size(); ++g) {
        const int nf = keys_i[g] / 32, kind = keys_i[g] % 32;
        if (smem_i.count(keys_i[g]) == 0) return fail(SST_EINTERNAL, "stream inverse group without its shared memory");
        const KernelTable *kt = table_for_nf(nf);
        int occ = 1;
        if (kt->occupancy(kind, smem_i[keys_i[g]], &occ) != cudaSuccess || occ < 1) occ = 1;
        const int grid = (int)std::min<int64_t>((int64_t)occ * sv->nsm, (int64_t)spans_i[g].second);
        cudaError_t e = kt->batch(kind, sv->d_ch, sv->d_items + spans_i[g].first, (int)spans_i[g].second, 0, grid,
                                  smem_i[keys_i[g]], nullptr, st);
        if (e != cudaSuccess) return cuda_fail(e, "stream inverse launch");
        count_launch();
    }
    if (!fin.empty()) {
        const int grid = (int)std::min<size_t>(fin.size(), (size_t)sv->nsm * 4);
        k_finalize_batch<<<grid, 256, 0, st>>>(sv->d_ch, sv->d_items + fin_off, (int)fin.size());
        SST_CU(cudaGetLastError(), "stream finalize launch");
        count_launch();
    }
    // 5. results back to the host
    size_t out_bytes = 0;
    for (auto &w : work) {
        Stream &S = sv->s[w.id];
        out_bytes += (S.xhat_only ? 0 : a256(sizeof(float2) * (size_t)(w.m_ready - S.m_next) * S.base.nbo)) +
                     a256(sizeof(float) * (size_t)(w.p_ready - S.p_next));
    }
    SST_CU(cudaStreamSynchronize(st), "tick");
    s = ensure_pinned(sv, out_bytes + 4096);
    if (s != SST_OK) return s;
    size_t o = 0;
    std::vector<std::pair<size_t, size_t>> where(work.size());
    for (size_t i = 0; i < work.size(); ++i) {
        Stream &S = sv->s[work[i].id];
        const int nbo = S.base.nbo;
        const size_t o_t = o;
        for (int64_t m = S.m_next; m < work[i].m_ready && !S.xhat_only;) {
            const int64_t r = m % S.trow_cap;
            const int64_t cnt = std::min<int64_t>(work[i].m_ready - m, S.trow_cap - r);
            SST_CU(cudaMemcpyAsync(sv->pin + o, S.T + (size_t)r * nbo, sizeof(float2) * (size_t)cnt * nbo,
                                   cudaMemcpyDeviceToHost, st), "TFR download");
            o += sizeof(float2) * (size_t)cnt * nbo;
            m += cnt;
        }
        o = a256(o);
        const size_t o_x = o;
        if (work[i].p_ready > S.p_next)
            SST_CU(cudaMemcpyAsync(sv->pin + o, S.xout, sizeof(float) * (size_t)(work[i].p_ready - S.p_next),
                                   cudaMemcpyDeviceToHost, st), "output download");
        o = a256(o + sizeof(float) * (size_t)(work[i].p_ready - S.p_next));
        where[i] = {o_t, o_x};
    }
    SST_CU(cudaStreamSynchronize(st), "tick");
    const double t_done = now_s();
    for (size_t i = 0; i < work.size(); ++i) {
        Stream &S = sv->s[work[i].id];
        const int nbo = S.base.nbo;
        const int64_t rows = work[i].m_ready - S.m_next;
        const float *tp = (const float *)(sv->pin + where[i].first);
        if (!S.xhat_only) S.tfr_host.insert(S.tfr_host.end(), tp, tp + 2 * (size_t)rows * nbo);
        const float *xp = (const float *)(sv->pin + where[i].second);
        S.x_host.insert(S.x_host.end(), xp, xp + (work[i].p_ready - S.p_next));
        for (double ta : work[i].arrivals) sv->lat.push_back(t_done - ta);
        S.m_next = work[i].m_ready;
        S.t_next = work[i].t_ready;
        S.p_next = work[i].p_ready;
        if (S.closing && S.p_next >= S.sig_end && S.m_next >= (S.sig_end + S.base.hop - 1) / S.base.hop) S.done = true;
    }
    return SST_OK;
}

SST_API sst_status sst_stream_poll(sst_service_t sv, int32_t id, float *tfr_host, int64_t max_cols, int64_t *cols,
                                   int64_t *first_col, float *xhat_host, int64_t max_samples, int64_t *samples,
                                   int64_t *first_sample, int32_t *finished) {
    SST_NVTX_RANGE();
    if (!sv) return fail(SST_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (id < 0 || id >= sv->max_streams || !sv->s[id].used) return fail(SST_EINVAL, "no open stream %d", id);
    Stream &S = sv->s[id];
    const int nbo = S.base.nbo;
    const int64_t have_c = (int64_t)S.tfr_host.size() / (2 * nbo);
    const int64_t nc = tfr_host ? std::min(have_c, max_cols) : 0;
    if (first_col) *first_col = S.tfr_first;
    if (nc > 0) {
        memcpy(tfr_host, S.tfr_host.data(), sizeof(float) * 2 * (size_t)nc * nbo);
        S.tfr_host.erase(S.tfr_host.begin(), S.tfr_host.begin() + 2 * (size_t)nc * nbo);
        S.tfr_first += nc;
    }
    if (cols) *cols = nc;
    const int64_t have_x = (int64_t)S.x_host.size();
    const int64_t nx = xhat_host ? std::min(have_x, max_samples) : 0;
    if (first_sample) *first_sample = S.x_first;
    if (nx > 0) {
        memcpy(xhat_host, S.x_host.data(), sizeof(float) * (size_t)nx);
        S.x_host.erase(S.x_host.begin(), S.x_host.begin() + nx);
        S.x_first += nx;
    }
    if (samples) *samples = nx;
    if (finished) *finished = (S.done && S.tfr_host.empty() && S.x_host.empty()) ? 1 : 0;
    return SST_OK;
}

SST_API sst_status sst_stream_release(sst_service_t sv, int32_t id) {
    if (!sv) return fail(SST_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (id < 0 || id >= sv->max_streams || !sv->s[id].used) return fail(SST_EINVAL, "no open stream %d", id);
    Stream &S = sv->s[id];
    cudaStreamSynchronize(sv->st);
    if (S.dmem) cudaFree(S.dmem);
    if (S.plan) sst_plan_destroy(S.plan);
    sv->used -= S.dev_bytes;
    sv->s[id] = Stream();
    return SST_OK;
}

SST_API sst_status sst_service_latency(sst_service_t sv, double *p50, double *p99, int64_t *count, int32_t reset) {
    if (!sv) return fail(SST_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    std::vector<double> v = sv->lat;
    if (count) *count = (int64_t)v.size();
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto q = [&](double f) { return v[std::min(v.size() - 1, (size_t)std::floor(f * (v.size() - 1) + 0.5))]; };
        if (p50) *p50 = q(0.50);
        if (p99) *p99 = q(0.99);
    } else {
        if (p50) *p50 = 0.0;
        if (p99) *p99 = 0.0;
    }
    if (reset) sv->lat.clear();
    return SST_OK;
}

SST_API sst_status sst_service_memory(sst_service_t sv, size_t *used, size_t *budget) {
    if (!sv) return fail(SST_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (used) *used = sv->used;
    if (budget) *budget = sv->budget;
    return SST_OK;
}

SST_API void sst_service_destroy(sst_service_t sv) {
    if (!sv) return;
    cudaStreamSynchronize(sv->st);
    for (auto &S : sv->s) {
        if (S.dmem) cudaFree(S.dmem);
        if (S.plan) sst_plan_destroy(S.plan);
    }
    if (sv->d_ch) cudaFree(sv->d_ch);
    if (sv->d_items) cudaFree(sv->d_items);
    if (sv->pin) cudaFreeHost(sv->pin);
    if (sv->st) cudaStreamDestroy(sv->st);
    delete sv;
}
