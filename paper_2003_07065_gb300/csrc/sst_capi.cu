// C ABI of libsst.so: plan creation (FP64 tables rounded to FP32), argument
// validation, workspace layout and the launch sequences of each entry point.
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sst_internal.h"
#include "sst_kernels.cuh"

namespace sst {

const KernelTable *table_nf_64();
const KernelTable *table_nf_128();
const KernelTable *table_nf_256();
const KernelTable *table_nf_512();
const KernelTable *table_nf_1024();
const KernelTable *table_nf_2048();
const KernelTable *table_nf_4096();
const KernelTable *table_nf_8192();

const KernelTable *table_for_nf(int nf) {
    switch (nf) {
        case 64: return table_nf_64();
        case 128: return table_nf_128();
        case 256: return table_nf_256();
        case 512: return table_nf_512();
        case 1024: return table_nf_1024();
        case 2048: return table_nf_2048();
        case 4096: return table_nf_4096();
        case 8192: return table_nf_8192();
    }
    return nullptr;
}

// ------------------------------------------------------------ small kernels
// Reduce the pre-pass partials (max |S^g|^2 per CTA for relative plans, max
// |x| per CTA for absolute ones) into the call's scalars (scalars_from_max).
__global__ void k_gamma(const float *__restrict__ partial, int count, float frac2, int from_x, float bound_mul,
                        int log2_nb, SstScalars *__restrict__ sc, float *__restrict__ maxv_out,
                        const unsigned *__restrict__ gate) {
    __shared__ float red[32];
    if (gate && *gate == 0u) return;
    float v = 0.f;
    for (int i = threadIdx.x; i < count; i += blockDim.x) v = fmaxf(v, partial[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float r = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, red[w]);
        *sc = scalars_from_max(r, frac2, from_x, bound_mul, log2_nb);
        if (maxv_out && !from_x) *maxv_out = sc->maxv;
    }
}

__global__ void k_absx(const float *__restrict__ x, int64_t n, float *__restrict__ partial) {
    __shared__ float red[32];
    float v = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v = fmaxf(v, fabsf(x[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float r = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, red[w]);
        partial[blockIdx.x] = r;
    }
}

cudaError_t launch_absx(const float *x, int64_t n, float *partial, int grid, cudaStream_t st) {
    k_absx<<<grid, 256, 0, st>>>(x, n, partial);
    return cudaGetLastError();
}

cudaError_t launch_gamma(const float *partial, int count, float frac2, int from_x, float bound_mul, int log2_nb,
                         SstScalars *sc, float *maxv_out, const unsigned *gate, cudaStream_t st) {
    k_gamma<<<1, 256, 0, st>>>(partial, count, frac2, from_x, bound_mul, log2_nb, sc, maxv_out, gate);
    return cudaGetLastError();
}

// ---- one-pass relative threshold (run_forward_spec)

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// max over frames of A_m = sum_j |x[m H + j - M]| |g_j|, which bounds |S^g| in
// every bin of frame m; folded into ctl[4] (float bits).  A CTA takes tiles
// of tf frames, staging the tile's |x| segment in shared memory ((tf + 2) H + L
// floats: a warp sums four consecutive frames at a time, and those past the
// tile's last read samples that are staged but not counted).
__global__ void k_frame_absmax(SstDev d, const float *__restrict__ x, int tf, unsigned *__restrict__ ctl) {
    extern __shared__ float seg[];
    __shared__ float red[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int64_t tiles = (d.F + tf - 1) / tf;
    const int len = (tf + 2) * d.hop + d.L;   // the tile's frames and three beyond (see below)
    float best = 0.f;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t m0 = t * tf;
        const int64_t s0 = m0 * d.hop - d.M;
        __syncthreads();
        for (int i = tid; i < len; i += blockDim.x) {
            const int64_t p = s0 + i;
            seg[i] = (p >= 0 && p < d.n) ? fabsf(x[p]) : 0.f;
        }
        __syncthreads();
        // four frames per warp at a time, sharing each load of |g|
        for (int f = 4 * warp; f < tf && m0 + f < d.F; f += 4 * nw) {
            const float *w = seg + f * d.hop;
            const int h = d.hop;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            for (int j = lane; j < d.L; j += 32) {
                const float gj = fabsf(__ldg(&d.g[j]));
                a0 = fmaf(w[j], gj, a0);
                a1 = fmaf(w[j + h], gj, a1);
                a2 = fmaf(w[j + 2 * h], gj, a2);
                a3 = fmaf(w[j + 3 * h], gj, a3);
            }
            a0 = warp_sum(a0);
            a1 = warp_sum(a1);
            a2 = warp_sum(a2);
            a3 = warp_sum(a3);
            // frames past the tile's (or the signal's) last read staged samples
            // that belong to no frame of the tile: only the tile's frames count
            const int64_t left = min((int64_t)tf - f, d.F - (m0 + f));
            best = fmaxf(best, a0);
            if (left > 1) best = fmaxf(best, a1);
            if (left > 2) best = fmaxf(best, a2);
            if (left > 3) best = fmaxf(best, a3);
        }
    }
    best = warp_max(best);
    if (lane == 0) red[warp] = best;
    __syncthreads();
    if (tid == 0) {
        float r = 0.f;
        for (int w = 0; w < nw; ++w) r = fmaxf(r, red[w]);
        if (r > 0.f) atomicMax(&ctl[4], __float_as_uint(r));
    }
}

// The one-pass scalars: g_lb2 from the sampled pre-pass maximum (a lower bound
// of max |S^g|^2, 0.1% margin against the two FFT packings' rounding), g_ub2
// and the fixed-point scale from max_m A_m (an upper bound, 0.1% margin).
__global__ void k_spec_scalars(const float *__restrict__ partial, int count, const unsigned *__restrict__ ctl,
                               float frac2, int log2_nb, SstScalars *__restrict__ sc) {
    __shared__ float red[32];
    float v = 0.f;
    for (int i = threadIdx.x; i < count; i += blockDim.x) v = fmaxf(v, partial[i]);
    v = warp_max(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float r = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, red[w]);
        const float amax = __uint_as_float(ctl[4]);
        SstScalars s = scalars_from_max(amax, frac2, 1, 1.001f, log2_nb);
        const float ub = amax * 1.001f;
        s.gamma2 = 0.f;
        s.maxv = 0.f;
        s.g_lb2 = frac2 * r * 0.999f;
        s.g_ub2 = frac2 * ub * ub;
        *sc = s;
    }
}

// Settle the waiting sources against the exact gamma^2 = frac^2 max |S^g|^2
// (the same arithmetic as k_gamma): a kept one adds its fixed-point value to
// its bin record (exact integer atomics, so the order does not matter).
__global__ void k_spec_fix_src(SpecBuf sb, const SstScalars *__restrict__ sc, float frac2) {
    if (sb.ctl[3]) return;
    const float gamma2 = frac2 * __uint_as_float(sb.ctl[0]);
    const unsigned n = min(sb.ctl[1], (unsigned)sb.cap_src);
    const float s1 = sc->s1, s2 = sc->s2;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const SpecSrc r = sb.src[i];
        if (r.bin < 0 || !(r.mag2 > gamma2)) continue;
        uint32_t alo, ahi, blo, bhi;   // as tacc_add
        tacc_split((r.vr * s1) * s2, alo, ahi);
        tacc_split((r.vi * s1) * s2, blo, bhi);
        uint32_t *w = sb.bin[r.bin].w;
        atomicAdd(&w[0], alo);
        atomicAdd(&w[1], ahi);
        atomicAdd(&w[2], blo);
        atomicAdd(&w[3], bhi);
    }
}

// Rewrite the T entries of the bins that received waiting sources.
__global__ void k_spec_fix_bin(SpecBuf sb, const SstScalars *__restrict__ sc, SstDev d, float2 *__restrict__ T) {
    if (sb.ctl[3]) return;
    const unsigned n = min(sb.ctl[2], (unsigned)sb.cap_bin);
    FwdScale fs;
    fs.r1 = sc->r1;
    fs.r2 = sc->r2;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const SpecBin r = sb.bin[i];
        if (r.l < 0) continue;   // an unused chunk tail
        T[(size_t)trow_of(d, r.m) * d.nbo + r.l] = make_float2(tacc_value(r.w[0], r.w[1], fs),
                                                               tacc_value(r.w[2], r.w[3], fs));
    }
}

// Settles the sources that the path without a TFR output deferred (those
// between the one-pass threshold's two bounds): a source above the exact
// gamma^2 = frac^2 max |S^g|^2 (the decision k_spec_fix_src takes) adds its
// share of the reconstruction to its tile's overlap-add segment, the
// coefficient's term of Eq. 25 times the window of Eq. 26,
// (g[n] / Nf) w 2 Re(S^g exp(2 pi i (z k_lo + l) n / (z Nf))) for |n| <= M,
// w = 1/2 at the coarse DC and Nyquist bins (their own Hermitian images).
// Sources are taken in the order of (frame, source bin) and each thread owns
// the segment samples tid + i SETTLE_T, so every sample's sum has a fixed
// order whatever order the records were taken in, and no barrier is needed
// between sources.  The phase steps along a thread's samples by one complex
// product.  One CTA per tile; shared memory: the segment, the window, then
// the records' keys and their order.
constexpr int SETTLE_T = 256;
__global__ void __launch_bounds__(SETTLE_T) k_fused_settle(SstDev d, float frac2, float *__restrict__ partial) {
    extern __shared__ float sseg[];
    if (d.spec.ctl[3]) return;   // a record list overflowed: the two-pass kernels redo the call
    const int tid = threadIdx.x;
    const int64_t tile = d.tile0 + blockIdx.x;
    const int n = d.fused_count[tile];
    if (n <= 0) return;
    float *gs = sseg + d.seg_len;
    int *key = reinterpret_cast<int *>(gs + d.L);
    int *ord = key + d.fused_cap;
    const SpecBin *rec = d.fused_rec + (size_t)tile * d.fused_cap;
    const int64_t m0 = tile * d.B;
    float *out = partial + (size_t)tslot_of(d, tile) * d.seg_len;
    const float cn = 2.0f / (float)d.nf;
    for (int i = tid; i < n; i += SETTLE_T) key[i] = (int)(rec[i].m - m0) * d.nb + (int)rec[i].w[3];
    for (int i = tid; i < d.seg_len; i += SETTLE_T) sseg[i] = out[i];
    for (int i = tid; i < d.L; i += SETTLE_T) gs[i] = __ldg(&d.g[i]) * cn;
    __syncthreads();
    for (int i = tid; i < n; i += SETTLE_T) {   // rank of each (unique) key
        const int k = key[i];
        int r = 0;
        for (int j = 0; j < n; ++j) r += key[j] < k;
        ord[r] = i;
    }
    __syncthreads();
    const float gamma2 = frac2 * __uint_as_float(d.spec.ctl[0]);
    const int zn = d.z * d.nf;
    const int ldc = (d.k_lo <= 0 && d.k_hi >= 0) ? -d.z * d.k_lo : -1;
    const int lnyq = (d.k_lo <= d.nf / 2 && d.k_hi >= d.nf / 2) ? d.z * (d.nf / 2 - d.k_lo) : -1;
    for (int r = 0; r < n; ++r) {
        const SpecBin b = rec[ord[r]];
        if (!(__uint_as_float(b.w[2]) > gamma2)) continue;
        const float w = (b.l == ldc || b.l == lnyq) ? 0.5f : 1.f;
        const float vr = __uint_as_float(b.w[0]) * w, vi = __uint_as_float(b.w[1]) * w;
        const int fz = d.z * d.k_lo + b.l;   // frequency in units of 1 / (z Nf)
        const int base = (int)(b.m - m0) * d.hop;   // segment index of the frame's tap -M
        // this thread's samples o = tid + i SETTLE_T in [base, base + L)
        int o = tid + ((base - tid + SETTLE_T - 1 > 0 ? base - tid + SETTLE_T - 1 : 0) / SETTLE_T) * SETTLE_T;
        if (o >= base + d.L) continue;
        const int t0 = o - base - d.M;   // n of the first sample
        int j = (int)(((long long)fz * t0) % zn);
        if (j < 0) j += zn;
        float2 e = __ldg(&d.twf[j]);
        const float2 E = __ldg(&d.twf[(int)(((long long)fz * SETTLE_T) % zn)]);
        for (int tt = o - base; tt < d.L; tt += SETTLE_T, o += SETTLE_T) {
            sseg[o] += gs[tt] * (vr * e.x - vi * e.y);
            e = make_float2(e.x * E.x - e.y * E.y, e.x * E.y + e.y * E.x);
        }
    }
    __syncthreads();
    for (int i = tid; i < d.seg_len; i += SETTLE_T) out[i] = sseg[i];
}

__global__ void k_finalize(SstDev d, const float *__restrict__ partial, float *__restrict__ xhat) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < d.n; p += (int64_t)gridDim.x * blockDim.x)
        xhat[p] = finalize_value(d, partial, p);
}

// The same, also storing every sample into a second buffer: page-locked host
// memory the device addresses directly (the end-to-end call's output, which
// then needs no copy of its own after the kernel).
__global__ void k_finalize_to(SstDev d, const float *__restrict__ partial, float *__restrict__ xhat,
                              float *__restrict__ xhat2) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < d.n; p += (int64_t)gridDim.x * blockDim.x) {
        const float v = finalize_value(d, partial, p);
        xhat[p] = v;
        xhat2[p] = v;
    }
}

// xhat[p - p0] for p in [p0, p1) (one part of a split signal)
__global__ void k_finalize_range(SstDev d, const float *__restrict__ partial, float *__restrict__ xhat, int64_t p0,
                                 int64_t p1) {
    for (int64_t p = p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < p1; p += (int64_t)gridDim.x * blockDim.x)
        xhat[p - p0] = finalize_value(d, partial, p);
}

// the largest of count pre-pass partial maxima
__global__ void k_reduce_max(const float *__restrict__ partial, int count, float *__restrict__ out) {
    __shared__ float red[32];
    float v = 0.f;
    for (int i = threadIdx.x; i < count; i += blockDim.x) v = fmaxf(v, partial[i]);
    v = warp_max(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float r = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, red[w]);
        *out = r;
    }
}

}  // namespace sst

using namespace sst;

// ------------------------------------------------------------ error state
namespace sst {
static thread_local std::string g_err;
static std::atomic<uint64_t> g_launches{0};

sst_status fail(sst_status s, const char *fmt, ...) {
    char b[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b, sizeof b, fmt, ap);
    va_end(ap);
    g_err = b;
    return s;
}

sst_status cuda_fail(cudaError_t e, const char *what) {
    return fail(SST_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static std::mutex g_smem_mu;
static std::map<std::pair<int, int>, size_t> g_smem_set;

cudaError_t raise_smem(const KernelTable *kt, int kind, size_t bytes) {
    std::lock_guard<std::mutex> lk(g_smem_mu);
    size_t &cur = g_smem_set[{kt->nf, kind}];
    if (bytes <= cur) return cudaSuccess;
    cudaError_t e = kt->set_smem(kind, bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

// ------------------------------------------------------------ profiling
static const char *kPkNames[SST_PROFILE_KINDS] = {"absmax", "gamma", "forward", "stft", "map", "inverse",
                                                  "finalize", "other", "fused"};
struct ProfRec { int kind; cudaEvent_t a, b; };
static std::mutex g_prof_mu;
static std::vector<ProfRec> g_prof;
static std::atomic<int> g_prof_on{0};

bool profiling_on() { return g_prof_on.load(std::memory_order_relaxed) != 0; }
void profile_record(int kind, cudaEvent_t a, cudaEvent_t b) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.push_back({kind, a, b});
}
}  // namespace sst

static int64_t round_half_up(double v) { return (int64_t)std::floor(v + 0.5); }
static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

static sst_status validate(const sst_params *p) {
    if (!p) return fail(SST_EINVAL, "params is NULL");
    if (p->n < 1) return fail(SST_EINVAL, "n must be >= 1 (got %lld)", (long long)p->n);
    if (!(p->fs > 0.0)) return fail(SST_EINVAL, "fs must be > 0");
    if (p->nfft < 64 || p->nfft > 8192 || (p->nfft & (p->nfft - 1)))
        return fail(SST_EINVAL, "nfft must be a power of two in [64, 8192] (got %d)", p->nfft);
    if (p->L < 3 || (p->L % 2) == 0) return fail(SST_EINVAL, "L must be odd and >= 3 (got %d)", p->L);
    if (p->L > SST_MAX_L) return fail(SST_EINVAL, "L must be <= %d (got %d)", SST_MAX_L, p->L);
    const int M = (p->L - 1) / 2;
    if (p->hop < 1 || p->hop > M) return fail(SST_EINVAL, "hop must be in [1, M = %d] (got %d)", M, p->hop);
    if (!(p->f_lo >= 0.0) || !(p->f_hi > p->f_lo) || p->f_hi > p->fs / 2 * (1 + 1e-12))
        return fail(SST_EINVAL, "band must satisfy 0 <= f_lo < f_hi <= fs/2");
    if (p->z < 1 || p->z > 16) return fail(SST_EINVAL, "z must be in [1, 16] (got %d)", p->z);
    if (!(p->gamma >= 0.0) || !std::isfinite(p->gamma)) return fail(SST_EINVAL, "gamma must be finite and >= 0");
    if ((p->g == nullptr) != (p->dg == nullptr)) return fail(SST_EINVAL, "give both g and dg, or neither");
    if (!p->g && !(p->sigma > 0.0)) return fail(SST_EINVAL, "sigma must be > 0 when g is not given");
    if (p->flags & ~(SST_GAMMA_RELATIVE | SST_TWO_PASS)) return fail(SST_EINVAL, "unknown flags 0x%x", p->flags);
    return SST_OK;
}

SST_API sst_status sst_plan_create(const sst_params *params, sst_plan_t *out) {
    SST_NVTX_RANGE();
    if (!out) return fail(SST_EINVAL, "out is NULL");
    *out = nullptr;
    sst_status st = validate(params);
    if (st != SST_OK) return st;
    const sst_params &p = *params;

    int dev = 0;
    SST_CU(cudaGetDevice(&dev), "cudaGetDevice");
    cudaDeviceProp prop;
    SST_CU(cudaGetDeviceProperties(&prop, dev), "cudaGetDeviceProperties");
    if (!(prop.major == 10 && prop.minor == 3))
        return fail(SST_EUNSUPPORTED, "libsst is built for sm_103a; device %d is sm_%d%d", dev, prop.major,
                    prop.minor);

    const KernelTable *kt = table_for_nf(p.nfft);
    if (!kt) return fail(SST_EINTERNAL, "no kernels for nfft %d", p.nfft);

    sst_plan *pl = new (std::nothrow) sst_plan();
    if (!pl) return fail(SST_ENOMEM, "host allocation failed");
    pl->p = p;
    pl->p.g = pl->p.dg = nullptr;
    pl->custom_window = params->g != nullptr;
    pl->device = dev;
    pl->num_sms = prop.multiProcessorCount;
    pl->kt = kt;

    const int L = p.L, M = (L - 1) / 2, nf = p.nfft, z = p.z, hop = p.hop;
    const int64_t n = p.n;
    const int64_t F = (n + hop - 1) / hop;
    int64_t k_lo = round_half_up(p.f_lo * nf / p.fs);
    int64_t k_hi = round_half_up(p.f_hi * nf / p.fs);
    if (k_hi > nf / 2) k_hi = nf / 2;
    if (k_lo > k_hi) k_lo = k_hi;
    const int nb = (int)(k_hi - k_lo + 1);
    const int nbo = z * (int)(k_hi - k_lo) + 1;

    // ---- FP64 tables
    std::vector<double> g(L), dg(L);
    if (params->g) {
        for (int i = 0; i < L; ++i) { g[i] = params->g[i]; dg[i] = params->dg[i]; }
    } else {
        const double amp = std::pow(M_PI * p.sigma * p.sigma, -0.25);
        for (int j = -M; j <= M; ++j) {
            const double v = amp * std::exp(-(double)j * j / (2.0 * p.sigma * p.sigma));
            g[j + M] = v;
            dg[j + M] = -((double)j / (p.sigma * p.sigma)) * v;
        }
    }
    if (!(g[M] > 0.0)) { delete pl; return fail(SST_EINVAL, "window must have g[0] > 0"); }
    const int G = z * nf;
    // inverse normaliser 1 / D[p], D[p] = g[0] sum_{m=0}^{F-1} g[p - m hop]  (Eq. 26)
    auto Dexact = [&](int64_t q) {
        int64_t mlo = (q - M > 0) ? (q - M + hop - 1) / hop : 0;
        int64_t mhi = (q + M) / hop;
        if (mhi > F - 1) mhi = F - 1;
        double s = 0.0;
        for (int64_t m = mlo; m <= mhi; ++m) {
            const int64_t j = q - m * hop;
            if (j >= -M && j <= M) s += g[j + M];
        }
        return g[M] * s;
    };
    const int64_t EL = std::min<int64_t>(n, M);
    const int64_t ER = std::max<int64_t>(EL, std::min<int64_t>(n, F * hop - M));
    std::vector<float> rDl(std::max<int64_t>(EL, 1)), rDr(std::max<int64_t>(n - ER, 1)), rDp(hop);
    for (int64_t q = 0; q < EL; ++q) rDl[q] = (float)(1.0 / Dexact(q));
    for (int64_t q = ER; q < n; ++q) rDr[q - ER] = (float)(1.0 / Dexact(q));
    for (int r = 0; r < hop; ++r) {
        double s = 0.0;
        for (int j = -M; j <= M; ++j)
            if ((((j % hop) + hop) % hop) == r) s += g[j + M];
        rDp[r] = (float)(1.0 / (g[M] * s));
    }
    for (int64_t q = 0; q < EL; ++q)
        if (!std::isfinite(rDl[q])) { delete pl; return fail(SST_EINVAL, "normaliser vanishes at sample %lld", (long long)q); }
    for (int64_t q = ER; q < n; ++q)
        if (!std::isfinite(rDr[q - ER])) { delete pl; return fail(SST_EINVAL, "normaliser vanishes at sample %lld", (long long)q); }

    // S^g' is packed as the imaginary part with the window s g', s = 2^round(log2(|g| / |g'|)),
    // so both halves of the packed FFT carry similar norms; 1/s is applied exactly afterwards
    double ng = 0.0, ndg = 0.0;
    for (int i = 0; i < L; ++i) { ng += g[i] * g[i]; ndg += dg[i] * dg[i]; }
    int sexp = (ndg > 0.0) ? (int)std::lround(0.5 * std::log2(ng / ndg)) : 0;
    if (sexp < -60) sexp = -60;
    if (sexp > 60) sexp = 60;
    const double dsc = std::ldexp(1.0, sexp);
    std::vector<float2> win(L);
    std::vector<float> gf(L);
    for (int i = 0; i < L; ++i) { win[i] = make_float2((float)g[i], (float)(dg[i] * dsc)); gf[i] = (float)g[i]; }
    pl->g64 = g;
    pl->dgs64.resize(L);
    for (int i = 0; i < L; ++i) pl->dgs64[i] = dg[i] * dsc;
    // second-order IF windows (built-in Gaussian only): g'' = (j^2 / sigma^4 -
    // 1 / sigma^2) g, t g = j g, t g' = j g', each scaled by a power of two
    // to the norm of g (undone exactly in the kernel)
    std::vector<float2> win2(L), win3(L);
    double s2 = 1.0, s3 = 1.0, s4 = 1.0;
    const bool so_ok = params->g == nullptr;
    if (so_ok) {
        std::vector<double> d2g(L), tg(L), tdg(L);
        double n2 = 0.0, n3 = 0.0, n4 = 0.0;
        const double sg2 = p.sigma * p.sigma;
        for (int i = 0; i < L; ++i) {
            const double j = (double)(i - M);
            d2g[i] = (j * j / (sg2 * sg2) - 1.0 / sg2) * g[i];
            tg[i] = j * g[i];
            tdg[i] = j * dg[i];
            n2 += d2g[i] * d2g[i];
            n3 += tg[i] * tg[i];
            n4 += tdg[i] * tdg[i];
        }
        auto eq = [&](double nh) {
            int e = nh > 0.0 ? (int)std::lround(0.5 * std::log2(ng / nh)) : 0;
            return std::ldexp(1.0, std::max(-60, std::min(60, e)));
        };
        s2 = eq(n2);
        s3 = eq(n3);
        s4 = eq(n4);
        for (int i = 0; i < L; ++i) {
            win2[i] = make_float2((float)(d2g[i] * s2), (float)(tg[i] * s3));
            win3[i] = make_float2((float)(tdg[i] * s4), 0.f);
        }
    }
    // Stockham twiddles, per radix-16 pass of span Ns (Ns = R1, 16 R1, ..., nf/16): rows
    // m = 1, 2, 4, 8 of exp(-2 pi i m k / (16 Ns)), k in [0, Ns), from entry 4 (Ns - R1) / 15
    int lg2 = 0;
    while ((1 << lg2) < nf) ++lg2;
    const int R1 = (lg2 % 4 == 0) ? 16 : (1 << (lg2 % 4));
    std::vector<float2> tw(std::max(4 * (nf - R1) / 15, 1));
    for (int Ns = R1; Ns < nf; Ns *= 16) {
        const int off = 4 * (Ns - R1) / 15;
        for (int mi = 0; mi < 4; ++mi)
            for (int k = 0; k < Ns; ++k) {
                const double a = -2.0 * M_PI * (double)(1 << mi) * (double)k / (16.0 * Ns);
                tw[off + mi * Ns + k] = make_float2((float)std::cos(a), (float)std::sin(a));
            }
    }
    // inverse sub-grid twiddles exp(+2 pi i s n / (z nf)), factored per last-pass output slot
    const int nsl = nf / 16;
    std::vector<float2> twb(z * nsl), twc(z * 32), twn(z);
    for (int s_ = 0; s_ < z; ++s_) {
        for (int j = 0; j < nsl; ++j) {
            const double a = 2.0 * M_PI * (double)s_ * (double)j / (double)G;
            twb[s_ * nsl + j] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
        for (int w = 0; w < 2; ++w)
            for (int r = 0; r < 16; ++r) {
                const double a = 2.0 * M_PI * (double)s_ * (double)r / (16.0 * z) - (w ? 2.0 * M_PI * (double)s_ / z : 0.0);
                twc[(2 * s_ + w) * 16 + r] = make_float2((float)std::cos(a), (float)std::sin(a));
            }
        const double a = -2.0 * M_PI * (double)s_ * (double)(nf / 2) / (double)G;
        twn[s_] = make_float2((float)std::cos(a), (float)std::sin(a));
    }

    // the settling pass's phases exp(2 pi i j / (z nf))
    std::vector<float2> twf((size_t)z * nf);
    for (int j = 0; j < z * nf; ++j) {
        const double a = 2.0 * M_PI * (double)j / (double)G;
        twf[j] = make_float2((float)std::cos(a), (float)std::sin(a));
    }

    // ---- one device allocation for all tables
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    const size_t o_win = take(sizeof(float2) * L), o_g = take(sizeof(float) * L),
                 o_tw = take(sizeof(float2) * tw.size()), o_twb = take(sizeof(float2) * twb.size()),
                 o_twc = take(sizeof(float2) * twc.size()), o_twn = take(sizeof(float2) * z),
                 o_rl = take(sizeof(float) * rDl.size()),
                 o_rr = take(sizeof(float) * rDr.size()), o_rp = take(sizeof(float) * hop),
                 o_w2 = take(sizeof(float2) * L), o_w3 = take(sizeof(float2) * L),
                 o_twf = take(sizeof(float2) * twf.size());
    cudaError_t ce = cudaMalloc(&pl->dmem, off);
    if (ce != cudaSuccess) { delete pl; return fail(SST_ENOMEM, "cudaMalloc of %zu table bytes failed", off); }
    char *base = (char *)pl->dmem;
    std::vector<char> host(off, 0);
    memcpy(host.data() + o_win, win.data(), sizeof(float2) * L);
    memcpy(host.data() + o_g, gf.data(), sizeof(float) * L);
    memcpy(host.data() + o_tw, tw.data(), sizeof(float2) * tw.size());
    memcpy(host.data() + o_twb, twb.data(), sizeof(float2) * twb.size());
    memcpy(host.data() + o_twc, twc.data(), sizeof(float2) * twc.size());
    memcpy(host.data() + o_twn, twn.data(), sizeof(float2) * z);
    memcpy(host.data() + o_rl, rDl.data(), sizeof(float) * rDl.size());
    memcpy(host.data() + o_rr, rDr.data(), sizeof(float) * rDr.size());
    memcpy(host.data() + o_rp, rDp.data(), sizeof(float) * hop);
    memcpy(host.data() + o_w2, win2.data(), sizeof(float2) * L);
    memcpy(host.data() + o_w3, win3.data(), sizeof(float2) * L);
    memcpy(host.data() + o_twf, twf.data(), sizeof(float2) * twf.size());
    ce = cudaMemcpy(base, host.data(), off, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) { cudaFree(pl->dmem); delete pl; return cuda_fail(ce, "table upload"); }

    SstDev &d = pl->d;
    d.win = (const float2 *)(base + o_win);
    d.g = (const float *)(base + o_g);
    d.tw = (const float2 *)(base + o_tw);
    d.twb = (const float2 *)(base + o_twb);
    d.twc = (const float2 *)(base + o_twc);
    d.twn = (const float2 *)(base + o_twn);
    d.twf = (const float2 *)(base + o_twf);
    d.rD_left = (const float *)(base + o_rl);
    d.rD_right = (const float *)(base + o_rr);
    d.rD_per = (const float *)(base + o_rp);
    d.n = n;
    d.F = F;
    d.EL = EL;
    d.ER = ER;
    d.L = L;
    d.M = M;
    d.hop = hop;
    d.nf = nf;
    d.z = z;
    d.k_lo = (int)k_lo;
    d.k_hi = (int)k_hi;
    d.nb = nb;
    d.nbo = nbo;
    int lg = 0;
    while ((1 << lg) < nb) ++lg;
    d.log2_nb = lg;
    d.c_if = (float)((double)nf / (2.0 * M_PI) / dsc);
    d.dscale = (float)(1.0 / dsc);
    d.win2 = so_ok ? (const float2 *)(base + o_w2) : nullptr;
    d.win3 = so_ok ? (const float2 *)(base + o_w3) : nullptr;
    d.r2 = (float)(1.0 / s2);
    d.r3 = (float)(1.0 / s3);
    d.r4 = (float)(1.0 / s4);
    d.c_so = (float)((double)nf / (2.0 * M_PI));
    d.relative = (p.flags & SST_GAMMA_RELATIVE) ? 1 : 0;
    d.gamma2_abs = d.relative ? 0.f : (float)(p.gamma * p.gamma);
    pl->gamma_frac2 = (float)(p.gamma * p.gamma);
    {
        double sg = 0.0;
        for (int i = 0; i < L; ++i) sg += std::fabs(g[i]);
        pl->sum_abs_g = (float)(sg * 1.001);
    }

    // inverse tiles: B even, enough tiles to fill the GPU several times over
    int64_t B = F / (4LL * pl->num_sms);
    if (B > 64) B = 64;
    if (B < 2) B = 2;
    B &= ~1LL;
    d.B = (int)B;
    d.seg_len = (int)((B - 1) * hop + L);
    d.ntiles = (F + B - 1) / B;

    // ---- shared memory and grids
    pl->smem_fwd_x = kt->smem_frame;
    // (forward kernels of class > 0 add the band's mirror values: below)
    pl->smem_fwd_t = kt->smem_frame + tacc_bytes(nbo);
    pl->smem_absmax = kt->smem_frame + sizeof(float2) * (kt->smem_frame - 128) / sizeof(float2);  // two frame buffers
    // inverse: frame buffer, the pair's two T rows regrouped by sub-grid, overlap-add segment
    pl->smem_inv = inverse_smem_bytes(kt->smem_frame, z, nb, d.seg_len);
    // pruned kernels where the band (and, for the forward, the window) leaves
    // part of the radix-16 first pass empty
    const int bcls = band_class(nf, kt->r1, (int)k_hi);
    const bool half_window = L <= nf / 2 + 1;
    const bool long_window = L > nf + 1;   // taps wrap more than once around the sub-grid transforms
    pl->inv_kind = half_window ? kind_cls(KIND_INV, bcls) : long_window ? KIND_INV_LONG : KIND_INV_WIDE;
    pl->kind_fwd_t = kind_cls(KIND_FWD_T, half_window ? bcls : 0);
    pl->kind_fwd_spec = kind_cls(KIND_FWD_SPEC, half_window ? bcls : 0);
    if (half_window && bcls > 0) pl->smem_fwd_t += mirror_bytes(nb);
    const size_t smax = prop.sharedMemPerBlockOptin;
    if (pl->smem_fwd_t > smax || pl->smem_inv > smax) {
        cudaFree(pl->dmem);
        delete pl;
        return fail(SST_EUNSUPPORTED, "shared memory need (%zu / %zu B) exceeds %zu B", pl->smem_fwd_t,
                    pl->smem_inv, smax);
    }
    pl->absmax_cls = half_window ? bcls : 0;
    struct { int kind; size_t bytes; } kinds[] = {{kind_cls(KIND_ABSMAX, pl->absmax_cls), pl->smem_absmax},
        {pl->kind_fwd_t, pl->smem_fwd_t},
        {KIND_FWD_STFT, pl->smem_fwd_x}, {KIND_FWD_MAP, pl->smem_fwd_x}, {pl->inv_kind, pl->smem_inv}};
    for (auto &k : kinds) {
        ce = raise_smem(kt, k.kind, k.bytes);
        if (ce != cudaSuccess) { cudaFree(pl->dmem); delete pl; return cuda_fail(ce, "cudaFuncSetAttribute"); }
    }
    auto grid_for = [&](int kind, size_t bytes, int64_t units) {
        int bl = 1;
        if (kt->occupancy(kind, bytes, &bl) != cudaSuccess || bl < 1) bl = 1;
        int64_t g_ = (int64_t)bl * pl->num_sms * 2;
        if (g_ > units) g_ = units;
        return (int)std::max<int64_t>(g_, 1);
    };
    // fused forward + inverse: the plan supports it where its shared memory fits
    pl->kind_fused = half_window ? kind_cls(KIND_FUSED, bcls) : long_window ? KIND_FUSED_LONG : KIND_FUSED_WIDE;
    pl->smem_fused = fused_smem_bytes(kt->smem_frame, nb, nbo, d.seg_len, half_window ? bcls : 0);
    pl->fused_ok = pl->smem_fused <= smax && raise_smem(kt, pl->kind_fused, pl->smem_fused) == cudaSuccess;
    pl->grid_absmax = grid_for(kind_cls(KIND_ABSMAX, pl->absmax_cls), pl->smem_absmax, (F + 3) / 4);
    pl->grid_fwd = grid_for(pl->kind_fwd_t, pl->smem_fwd_t, F);
    pl->grid_fwd_x = grid_for(KIND_FWD_STFT, pl->smem_fwd_x, F);

    // Forwards of class 1 or 2 keep their band values in registers, so the
    // frame buffer is free between the last FFT pass and the next frame: the
    // T accumulators go there (k_forward_alias), a third of the shared memory
    // and four CTAs per SM instead of three, where they fit in the buffer.
    const int frame_buf = (int)((kt->smem_frame - 128) / sizeof(float2));
    const bool fwd_alias = half_window && bcls > 0 && kt->r1 == 16 && tacc_fits_frame(nbo, frame_buf);
    // its chunks of consecutive frames (staged samples): up to 16 frames, at
    // least about eight chunks per CTA
    d.fwd_chunk = (int)std::max<int64_t>(1, std::min<int64_t>(16, F / (8LL * pl->num_sms)));
    const int seg_floats = fwd_seg_floats(d.fwd_chunk, hop, L);
    const int64_t fwd_chunks = (F + d.fwd_chunk - 1) / d.fwd_chunk;

    // ---- one-pass relative threshold (default for relative plans)
    pl->smem_fwd_spec = pl->smem_fwd_t +
                        (spec_in_frame(nb, nbo, (int)((kt->smem_frame - 128) / sizeof(float2))) ? 0 : spec_smem_bytes(nbo));
    // frames per tile of the A_m bound (k_frame_absmax): its segment of
    // (tf + 2) H + L floats within 48 KiB where it can be, else one frame per
    // tile with the kernel's shared-memory limit raised
    pl->spec_tf = (int)std::max<int64_t>(1, std::min<int64_t>(32, (12000 - (int64_t)L) / hop - 2));
    pl->smem_frame_absmax = sizeof(float) * ((size_t)(pl->spec_tf + 2) * hop + L);
    bool bound_ok = pl->smem_frame_absmax <= 48 * 1024;
    if (!bound_ok && pl->smem_frame_absmax <= smax)
        bound_ok = cudaFuncSetAttribute(k_frame_absmax, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)pl->smem_frame_absmax) == cudaSuccess;
    pl->spec = d.relative && !(p.flags & SST_TWO_PASS) && pl->smem_fwd_spec <= smax && bound_ok;
    if (pl->spec) {
        ce = raise_smem(kt, pl->kind_fwd_spec, pl->smem_fwd_spec);
        if (ce != cudaSuccess) { cudaFree(pl->dmem); delete pl; return cuda_fail(ce, "cudaFuncSetAttribute"); }
        pl->grid_fwd_spec = grid_for(pl->kind_fwd_spec, pl->smem_fwd_spec, F);
        if (fwd_alias) {   // (see below)
            const int ka = kind_cls(KIND_FWD_SPECA, bcls);
            const size_t ba = forward_alias_smem_bytes(frame_buf, nb, true, seg_floats);
            if (ba <= smax && raise_smem(kt, ka, ba) == cudaSuccess) {
                pl->kind_fwd_spec = ka;
                pl->smem_fwd_spec = ba;
                pl->grid_fwd_spec = grid_for(ka, ba, fwd_chunks);
            }
        }
        // records: 1/64 of the sources, plus the chunk tails each CTA may leave unused
        pl->spec_cap = (int)std::min<int64_t>(std::max<int64_t>(4096, F * (int64_t)nb / 64) +
                                                  (int64_t)SPEC_CHUNK * pl->grid_fwd_spec,
                                              (int64_t)1 << 28);
        // the path without a TFR output records its waiting sources per
        // inverse tile: room for 1/32 of a tile's sources (64 .. 2048)
        if (pl->fused_ok) {
            const int cap = (int)std::max<int64_t>(64, std::min<int64_t>(2048, (int64_t)d.B * nb / 32));
            const size_t sm = sizeof(float) * ((size_t)d.seg_len + L) + 2 * sizeof(int) * (size_t)cap;
            bool ok = true;
            if (ok && sm > 48 * 1024)
                ok = sm <= smax && cudaFuncSetAttribute(k_fused_settle, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        (int)sm) == cudaSuccess;
            pl->fused_spec = ok;
            pl->fused_cap = cap;
            pl->smem_settle = sm;
        }
    }

    if (fwd_alias) {
        const int ka = kind_cls(KIND_FWD_TA, bcls);
        const size_t ba = forward_alias_smem_bytes(frame_buf, nb, false, seg_floats);
        if (ba <= smax && raise_smem(kt, ka, ba) == cudaSuccess) {
            pl->kind_fwd_t = ka;
            pl->smem_fwd_t = ba;
            pl->grid_fwd = grid_for(ka, ba, fwd_chunks);
        }
    }

    // ---- workspace: [scalars 256 B][absmax partials][overlap-add partials]
    //      then, for the one-pass threshold, [control 256 B][source records][bin records]
    //      and, for its path without a TFR output, [per-tile records][per-tile counts]
    pl->ws_off_partial = 256;
    pl->ws_off_ola = align256(pl->ws_off_partial + sizeof(float) * pl->grid_absmax);
    pl->ws_bytes = align256(pl->ws_off_ola + sizeof(float) * (size_t)d.ntiles * d.seg_len);
    if (pl->spec) {
        pl->ws_off_spec = pl->ws_bytes;
        pl->ws_bytes = align256(pl->ws_off_spec + 256 + (sizeof(SpecSrc) + sizeof(SpecBin)) * (size_t)pl->spec_cap);
    }
    if (pl->fused_spec) {   // [per-tile records][per-tile counts]
        pl->ws_off_fused = pl->ws_bytes;
        pl->ws_bytes = align256(pl->ws_off_fused + sizeof(SpecBin) * (size_t)pl->fused_cap * (size_t)d.ntiles +
                                sizeof(int32_t) * (size_t)d.ntiles);
    }
    *out = pl;
    return SST_OK;
}

SST_API void sst_plan_destroy(sst_plan_t plan) {
    if (!plan) return;
    if (plan->dmem) cudaFree(plan->dmem);
    delete plan;
}

SST_API sst_status sst_plan_query(sst_plan_t plan, int64_t *frames, int32_t *bins, int32_t *k_lo, int32_t *k_hi,
                                  size_t *workspace_bytes) {
    if (!plan) return fail(SST_EINVAL, "plan is NULL");
    if (frames) *frames = plan->d.F;
    if (bins) *bins = plan->d.nbo;
    if (k_lo) *k_lo = plan->d.k_lo;
    if (k_hi) *k_hi = plan->d.k_hi;
    if (workspace_bytes) *workspace_bytes = plan->ws_bytes;
    return SST_OK;
}

// ------------------------------------------------------------ parameter guard
// Sec. 4: Eq. 35 (sigma_f), Eq. 37-38 and Eq. 46 (bounds on Hf = n / nfft).
// sigma_samples is the window's standard deviation in samples.
static void guard_report(const sst_params &p, double sigma_samples, sst_param_report *out) {
    sst_param_report r;
    memset(&r, 0, sizeof r);
    r.sigma_s = sigma_samples / p.fs;
    r.sigma_f_hz = 1.0 / (2.0 * M_PI * r.sigma_s);
    r.hf = (double)p.n / (double)p.nfft;
    r.hf_max_eq38 = 3.0 * (double)p.n / (4.0 * M_PI * r.sigma_s * p.fs);
    r.hf_max_eq46 = std::sqrt(2.0) * r.sigma_f_hz * (double)p.n / p.fs;
    r.delta_f_hz = p.fs / (double)p.nfft;
    r.delta_f_fine_hz = p.fs / ((double)p.nfft * (double)p.z);
    r.delta_f_max_eq37_hz = 1.5 * r.sigma_f_hz;
    r.delta_f_max_eq46_hz = std::sqrt(2.0) * r.sigma_f_hz;
    if (r.hf >= r.hf_max_eq38) r.flags |= SST_GUARD_EQ38;
    if (r.hf >= r.hf_max_eq46) r.flags |= SST_GUARD_EQ46;
    *out = r;
}

// standard deviation (samples) of a window: sqrt(2 sum j^2 g^2 / sum g^2),
// which is sigma for g proportional to exp(-j^2 / (2 sigma^2))
static double window_sigma(const double *g, int L) {
    const int M = (L - 1) / 2;
    double s0 = 0.0, s2 = 0.0;
    for (int i = 0; i < L; ++i) {
        const double j = (double)(i - M), e = g[i] * g[i];
        s0 += e;
        s2 += j * j * e;
    }
    return s0 > 0.0 ? std::sqrt(2.0 * s2 / s0) : 0.0;
}

SST_API sst_status sst_params_check(const sst_params *params, sst_param_report *out) {
    if (!out) return fail(SST_EINVAL, "out is NULL");
    sst_status st = validate(params);
    if (st != SST_OK && st != SST_EUNSUPPORTED) return st;
    const double sig = params->g ? window_sigma(params->g, params->L) : params->sigma;
    if (!(sig > 0.0)) return fail(SST_EINVAL, "the window has no spread (sum of g^2 is zero)");
    guard_report(*params, sig, out);
    return SST_OK;
}

SST_API sst_status sst_plan_check(sst_plan_t plan, sst_param_report *out) {
    if (!plan) return fail(SST_EINVAL, "plan is NULL");
    if (!out) return fail(SST_EINVAL, "out is NULL");
    const double sig = plan->custom_window ? window_sigma(plan->g64.data(), plan->p.L) : plan->p.sigma;
    if (!(sig > 0.0)) return fail(SST_EINVAL, "the window has no spread (sum of g^2 is zero)");
    guard_report(plan->p, sig, out);
    return SST_OK;
}

// ------------------------------------------------------------ launches
static sst_status check_call(sst_plan_t plan, const void *x, int64_t n, const void *ws) {
    if (!plan) return fail(SST_EINVAL, "plan is NULL");
    if (!x) return fail(SST_EINVAL, "input pointer is NULL");
    if (n != plan->d.n) return fail(SST_EINVAL, "n = %lld differs from the plan's n = %lld", (long long)n,
                                    (long long)plan->d.n);
    if (!ws) return fail(SST_EINVAL, "workspace is NULL");
    if (((uintptr_t)ws) & 255) return fail(SST_EINVAL, "workspace must be 256-byte aligned");
    int dev = -1;
    SST_CU(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != plan->device) return fail(SST_EINVAL, "plan was created on device %d, current is %d", plan->device, dev);
    return SST_OK;
}

static SstScalars *ws_scalars(sst_plan_t, void *ws) { return (SstScalars *)ws; }
static float *ws_partial(sst_plan_t pl, void *ws) { return (float *)((char *)ws + pl->ws_off_partial); }
static float *ws_ola(sst_plan_t pl, void *ws) { return (float *)((char *)ws + pl->ws_off_ola); }
// the call's status word (SST_DEV_*: a bounded wait of a staged copy gave
// up), in the workspace's 256-byte header; cleared at the start of every
// entry point that runs the forward or the inverse, read by sst_check
static unsigned *ws_status(sst_plan_t, void *ws) { return (unsigned *)((char *)ws + 192); }
static sst_status clear_status(sst_plan_t pl, void *ws, cudaStream_t st) {
    SST_CU(cudaMemsetAsync(ws_status(pl, ws), 0, sizeof(unsigned), st), "status reset");
    return SST_OK;
}

// The pre-pass of a forward call: for relative plans the max |S^g| pre-pass,
// for absolute plans a max |x| reduction (only needed for the T scale).
// Fills the SstScalars at sc; partial holds grid_absmax floats.
static sst_status run_prepass(sst_plan_t pl, const float *x, SstScalars *sc, float *partial, cudaStream_t st,
                              float *maxv_out, bool profile = true) {
    if (pl->d.relative) {
        cudaError_t e;
        if (profile) {
            SST_LAUNCHED_K(PK_ABSMAX, st, pl->kt->absmax(pl->d, pl->absmax_cls, x, partial, pl->grid_absmax, pl->smem_absmax, st),
                           "absmax launch");
        } else {
            e = pl->kt->absmax(pl->d, pl->absmax_cls, x, partial, pl->grid_absmax, pl->smem_absmax, st);
            if (e != cudaSuccess) return cuda_fail(e, "absmax launch");
            count_launch();
        }
    } else {
        int64_t blocks = (pl->d.n + 255) / 256;
        if (blocks > pl->grid_absmax) blocks = pl->grid_absmax;
        k_absx<<<(unsigned)blocks, 256, 0, st>>>(x, pl->d.n, partial);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "absx launch");
        count_launch();
    }
    const int count = pl->d.relative ? pl->grid_absmax
                                     : (int)std::min<int64_t>((pl->d.n + 255) / 256, pl->grid_absmax);
    if (profile) {
        SST_LAUNCHED_K(PK_GAMMA, st,
                       (k_gamma<<<1, 256, 0, st>>>(partial, count, pl->gamma_frac2, pl->d.relative ? 0 : 1,
                                                   pl->sum_abs_g, pl->d.log2_nb, sc, maxv_out, nullptr),
                        cudaGetLastError()),
                       "gamma launch");
    } else {
        k_gamma<<<1, 256, 0, st>>>(partial, count, pl->gamma_frac2, pl->d.relative ? 0 : 1, pl->sum_abs_g,
                                   pl->d.log2_nb, sc, maxv_out, nullptr);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "gamma launch");
        count_launch();
    }
    return SST_OK;
}

static SpecBuf ws_spec(sst_plan_t pl, void *ws) {
    SpecBuf b;
    char *base = (char *)ws + pl->ws_off_spec;
    b.ctl = (unsigned *)base;
    b.src = (SpecSrc *)(base + 256);
    b.bin = (SpecBin *)(base + 256 + sizeof(SpecSrc) * (size_t)pl->spec_cap);
    b.cap_src = b.cap_bin = pl->spec_cap;
    return b;
}

// Relative threshold in one forward pass.  The FFT pre-pass over every frame
// (about a third of the forward's cost) is replaced by two cheap bounds:
// g_lb from the pre-pass on every 16th group of four frames (below the true
// gamma), g_ub from max_m A_m (above it).  The forward keeps sources above
// g_ub at once, drops those at or below g_lb, and records the rest with the
// exact partial sums of their bins; it also finds the exact max |S^g|.  Two
// small kernels then keep the recorded sources above the exact gamma and
// rewrite their bins.  Same kept set and the same exact sums as the two-pass
// path (up to the rounding of max |S^g|).  If a record buffer overflows, the
// two-pass kernels, launched behind a device-side gate, redo the forward.
static constexpr int kSpecStride = 16;
// The one-pass threshold's bounds and scalars: the control words cleared,
// max_m A_m (k_frame_absmax), the sampled pre-pass, then g_lb2, g_ub2 and the
// fixed-point scale (k_spec_scalars).
static sst_status run_spec_bounds(sst_plan_t pl, const SstDev &d, const float *x, void *ws, cudaStream_t st) {
    SstScalars *sc = ws_scalars(pl, ws);
    float *partial = ws_partial(pl, ws);
    const SpecBuf sb = ws_spec(pl, ws);
    SST_CU(cudaMemsetAsync(sb.ctl, 0, 64, st), "control reset");
    {
        const int64_t tiles = (d.F + pl->spec_tf - 1) / pl->spec_tf;
        const int grid = (int)std::min<int64_t>(tiles, (int64_t)pl->num_sms * 8);
        const size_t smem = pl->smem_frame_absmax;
        SST_LAUNCHED_K(PK_ABSMAX, st,
                       (k_frame_absmax<<<grid, 256, smem, st>>>(d, x, pl->spec_tf, sb.ctl), cudaGetLastError()),
                       "frame bound launch");
    }
    SstDev ds = d;
    ds.sample_stride = kSpecStride;
    SST_LAUNCHED_K(PK_ABSMAX, st, pl->kt->absmax(ds, pl->absmax_cls, x, partial, pl->grid_absmax, pl->smem_absmax, st),
                   "sampled pre-pass launch");
    SST_LAUNCHED_K(PK_GAMMA, st,
                   (k_spec_scalars<<<1, 256, 0, st>>>(partial, pl->grid_absmax, sb.ctl, pl->gamma_frac2, d.log2_nb,
                                                      sc),
                    cudaGetLastError()),
                   "one-pass scalars launch");
    return SST_OK;
}

static sst_status run_forward_spec(sst_plan_t pl, const SstDev &d, const float *x, float *tfr, void *ws,
                                   cudaStream_t st) {
    SstScalars *sc = ws_scalars(pl, ws);
    float *partial = ws_partial(pl, ws);
    const SpecBuf sb = ws_spec(pl, ws);
    sst_status s = run_spec_bounds(pl, d, x, ws, st);
    if (s != SST_OK) return s;
    SstDev df = d;
    df.spec = sb;
    SST_LAUNCHED_K(PK_FORWARD, st,
                   pl->kt->forward(df, pl->kind_fwd_spec, x, sc, tfr, nullptr, pl->grid_fwd_spec, pl->smem_fwd_spec, st),
                   "one-pass forward launch");
    const int gfix = pl->num_sms * 4;
    SST_LAUNCHED_K(PK_OTHER, st, (k_spec_fix_src<<<gfix, 256, 0, st>>>(sb, sc, pl->gamma_frac2), cudaGetLastError()),
                   "threshold settle launch");
    SST_LAUNCHED_K(PK_OTHER, st, (k_spec_fix_bin<<<gfix, 256, 0, st>>>(sb, sc, d, (float2 *)tfr), cudaGetLastError()),
                   "bin rewrite launch");
    // the two-pass path, run only if a record buffer overflowed
    SstDev dg = d;
    dg.gate = sb.ctl + 3;
    SST_LAUNCHED_K(PK_ABSMAX, st, pl->kt->absmax(dg, pl->absmax_cls, x, partial, pl->grid_absmax, pl->smem_absmax, st),
                   "absmax launch");
    SST_LAUNCHED_K(PK_GAMMA, st,
                   (k_gamma<<<1, 256, 0, st>>>(partial, pl->grid_absmax, pl->gamma_frac2, 0, 1.f, d.log2_nb, sc,
                                               nullptr, sb.ctl + 3),
                    cudaGetLastError()),
                   "gamma launch");
    SST_LAUNCHED_K(PK_FORWARD, st,
                   pl->kt->forward(dg, pl->kind_fwd_t, x, sc, tfr, nullptr, pl->grid_fwd, pl->smem_fwd_t, st),
                   "forward launch");
    return SST_OK;
}

static sst_status run_forward(sst_plan_t pl, const float *x, float *tfr, void *ws, cudaStream_t st) {
    SstDev d = pl->d;
    d.status = ws_status(pl, ws);
    d.test_withhold = pl->test_withhold_fwd.exchange(0) ? 1 : 0;
    if (pl->spec) return run_forward_spec(pl, d, x, tfr, ws, st);
    sst_status s = run_prepass(pl, x, ws_scalars(pl, ws), ws_partial(pl, ws), st, nullptr);
    if (s != SST_OK) return s;
    SST_LAUNCHED_K(PK_FORWARD, st,
                   pl->kt->forward(d, pl->kind_fwd_t, x, ws_scalars(pl, ws), tfr, nullptr, pl->grid_fwd, pl->smem_fwd_t, st),
                   "forward launch");
    return SST_OK;
}


// xhat[p] (and xhat2[p], if not null) from the overlap-add partials
static sst_status launch_finalize(sst_plan_t pl, float *xhat, float *xhat2, void *ws, cudaStream_t st) {
    int64_t blocks = (pl->d.n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (xhat2) {
        SST_LAUNCHED_K(PK_FINALIZE, st,
                       (k_finalize_to<<<(unsigned)blocks, 256, 0, st>>>(pl->d, ws_ola(pl, ws), xhat, xhat2),
                        cudaGetLastError()),
                       "finalize launch");
    } else {
        SST_LAUNCHED_K(PK_FINALIZE, st,
                       (k_finalize<<<(unsigned)blocks, 256, 0, st>>>(pl->d, ws_ola(pl, ws), xhat), cudaGetLastError()),
                       "finalize launch");
    }
    return SST_OK;
}

static sst_status run_inverse(sst_plan_t pl, const float *tfr, float *xhat, void *ws, cudaStream_t st,
                              const int32_t *zone = nullptr, int zone_hw = 0, float *xhat2 = nullptr) {
    SstDev d = pl->d;
    d.zone = zone;
    d.zone_hw = zone_hw;
    d.status = ws_status(pl, ws);
    d.test_withhold = pl->test_withhold.exchange(0) ? 1 : 0;
    SST_LAUNCHED_K(PK_INVERSE, st, pl->kt->inverse(d, pl->inv_kind, (const float2 *)tfr, ws_ola(pl, ws), pl->smem_inv, st),
                   "inverse launch");
    return launch_finalize(pl, xhat, xhat2, ws, st);
}


SST_API sst_status sst_forward(sst_plan_t plan, const float *x_dev, int64_t n, float *tfr_dev, void *ws, void *stream) {
    SST_NVTX_RANGE();
    sst_status s = check_call(plan, x_dev, n, ws);
    if (s != SST_OK) return s;
    if (!tfr_dev) return fail(SST_EINVAL, "tfr pointer is NULL");
    s = clear_status(plan, ws, (cudaStream_t)stream);
    if (s != SST_OK) return s;
    return run_forward(plan, x_dev, tfr_dev, ws, (cudaStream_t)stream);
}

SST_API sst_status sst_inverse(sst_plan_t plan, const float *tfr_dev, int64_t n, float *xhat_dev, void *ws,
                               void *stream) {
    SST_NVTX_RANGE();
    sst_status s = check_call(plan, tfr_dev, n, ws);
    if (s != SST_OK) return s;
    if (!xhat_dev) return fail(SST_EINVAL, "xhat pointer is NULL");
    s = clear_status(plan, ws, (cudaStream_t)stream);
    if (s != SST_OK) return s;
    return run_inverse(plan, tfr_dev, xhat_dev, ws, (cudaStream_t)stream);
}

SST_API sst_status sst_inverse_zone(sst_plan_t plan, const float *tfr_dev, int64_t n, const int32_t *ridge_dev,
                                    int32_t half_width, float *xhat_dev, void *ws, void *stream) {
    SST_NVTX_RANGE();
    sst_status s = check_call(plan, tfr_dev, n, ws);
    if (s != SST_OK) return s;
    if (!xhat_dev) return fail(SST_EINVAL, "xhat pointer is NULL");
    if (!ridge_dev) return fail(SST_EINVAL, "ridge pointer is NULL");
    if (((uintptr_t)ridge_dev) & 3) return fail(SST_EINVAL, "ridge must be 4-byte aligned");
    if (half_width < 0 || half_width > (1 << 28)) return fail(SST_EINVAL, "half_width = %d out of range", half_width);
    s = clear_status(plan, ws, (cudaStream_t)stream);
    if (s != SST_OK) return s;
    return run_inverse(plan, tfr_dev, xhat_dev, ws, (cudaStream_t)stream, ridge_dev, half_width);
}

// Forward + inverse with T kept on chip (k_fused): the pre-pass (relative
// plans: max |S^g| over every frame, as SST_TWO_PASS plans do, since no T
// exists to settle afterwards), one fused launch over the inverse tiles, and
// k_finalize.
// The path without a TFR output with the one-pass relative threshold: the
// bounds, k_fused (sources between them left out of the rows and recorded
// per tile, the exact max |S^g| found), k_fused_settle (the recorded sources
// the exact gamma keeps added to the segments); should a tile's records
// overflow, the two-pass kernels behind the gate word redo the call.
static sst_status run_fused_spec(sst_plan_t pl, const float *x, void *ws, cudaStream_t st) {
    const SstDev &d = pl->d;
    SstScalars *sc = ws_scalars(pl, ws);
    float *partial = ws_partial(pl, ws);
    const SpecBuf sb = ws_spec(pl, ws);
    sst_status s = run_spec_bounds(pl, d, x, ws, st);
    if (s != SST_OK) return s;
    SstDev df = d;
    df.spec = sb;
    df.fused_rec = reinterpret_cast<SpecBin *>((char *)ws + pl->ws_off_fused);
    df.fused_count = reinterpret_cast<int32_t *>(df.fused_rec + (size_t)pl->fused_cap * d.ntiles);
    df.fused_cap = pl->fused_cap;
    SST_LAUNCHED_K(PK_FUSED, st, pl->kt->fused(df, pl->kind_fused, x, sc, ws_ola(pl, ws), pl->smem_fused, st),
                   "fused launch");
    SST_LAUNCHED_K(PK_OTHER, st,
                   (k_fused_settle<<<(unsigned)d.ntiles, SETTLE_T, pl->smem_settle, st>>>(df, pl->gamma_frac2,
                                                                                     ws_ola(pl, ws)),
                    cudaGetLastError()),
                   "settle launch");
    SstDev dg = d;
    dg.gate = sb.ctl + 3;
    SST_LAUNCHED_K(PK_ABSMAX, st, pl->kt->absmax(dg, pl->absmax_cls, x, partial, pl->grid_absmax, pl->smem_absmax, st),
                   "absmax launch");
    SST_LAUNCHED_K(PK_GAMMA, st,
                   (k_gamma<<<1, 256, 0, st>>>(partial, pl->grid_absmax, pl->gamma_frac2, 0, 1.f, d.log2_nb, sc,
                                               nullptr, sb.ctl + 3),
                    cudaGetLastError()),
                   "gamma launch");
    SST_LAUNCHED_K(PK_FUSED, st, pl->kt->fused(dg, pl->kind_fused, x, sc, ws_ola(pl, ws), pl->smem_fused, st),
                   "fused launch");
    return SST_OK;
}

static sst_status run_fused(sst_plan_t pl, const float *x, float *xhat, void *ws, cudaStream_t st,
                            float *xhat2 = nullptr) {
    if (pl->fused_spec) {
        sst_status s = run_fused_spec(pl, x, ws, st);
        if (s != SST_OK) return s;
    } else {
        sst_status s = run_prepass(pl, x, ws_scalars(pl, ws), ws_partial(pl, ws), st, nullptr);
        if (s != SST_OK) return s;
        SST_LAUNCHED_K(PK_FUSED, st,
                       pl->kt->fused(pl->d, pl->kind_fused, x, ws_scalars(pl, ws), ws_ola(pl, ws), pl->smem_fused, st),
                       "fused launch");
    }
    return launch_finalize(pl, xhat, xhat2, ws, st);
}

// sst_forward_inverse, the reconstruction also stored into xhat2 when not null
static sst_status forward_inverse_to(sst_plan_t plan, const float *x_dev, int64_t n, float *tfr_dev,
                                     float *xhat_dev, float *xhat2, void *ws, void *stream) {
    sst_status s = check_call(plan, x_dev, n, ws);
    if (s != SST_OK) return s;
    if (!xhat_dev) return fail(SST_EINVAL, "xhat pointer is NULL");
    if (!tfr_dev) {
        if (!plan->fused_ok)
            return fail(SST_EUNSUPPORTED,
                        "no TFR output needs the fused kernel, whose %zu bytes of shared memory this plan exceeds",
                        plan->smem_fused);
        return run_fused(plan, x_dev, xhat_dev, ws, (cudaStream_t)stream, xhat2);
    }
    s = clear_status(plan, ws, (cudaStream_t)stream);
    if (s != SST_OK) return s;
    s = run_forward(plan, x_dev, tfr_dev, ws, (cudaStream_t)stream);
    if (s != SST_OK) return s;
    return run_inverse(plan, tfr_dev, xhat_dev, ws, (cudaStream_t)stream, nullptr, 0, xhat2);
}

SST_API sst_status sst_forward_inverse(sst_plan_t plan, const float *x_dev, int64_t n, float *tfr_dev,
                                       float *xhat_dev, void *ws, void *stream) {
    SST_NVTX_RANGE();
    return forward_inverse_to(plan, x_dev, n, tfr_dev, xhat_dev, nullptr, ws, stream);
}

SST_API sst_status sst_forward_inverse_host(sst_plan_t plan, const float *x_host, int64_t n, float *xhat_host,
                                            float *x_dev, float *tfr_dev, float *xhat_dev, void *ws, void *stream) {
    SST_NVTX_RANGE();
    if (!x_host || !xhat_host) return fail(SST_EINVAL, "host pointer is NULL");
    sst_status s = check_call(plan, x_dev, n, ws);
    if (s != SST_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // an output in page-locked memory that the device addresses is written
    // by the finalising kernel itself (no copy after it)
    float *direct = nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, xhat_host) == cudaSuccess) {
        if (at.type == cudaMemoryTypeHost && at.devicePointer) direct = (float *)at.devicePointer;
    } else {
        (void)cudaGetLastError();   // (pageable memory: not an error)
    }
    SST_CU(cudaMemcpyAsync(x_dev, x_host, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, st), "input copy");
    s = forward_inverse_to(plan, x_dev, n, tfr_dev, xhat_dev, direct, ws, stream);
    if (s != SST_OK) return s;
    if (!direct)
        SST_CU(cudaMemcpyAsync(xhat_host, xhat_dev, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, st),
               "output copy");
    SST_CU(cudaStreamSynchronize(st), "stream synchronise");
    return SST_OK;
}

SST_API sst_status sst_stft(sst_plan_t plan, const float *x_dev, int64_t n, float *V_dev, float *Vd_dev, void *ws,
                            void *stream) {
    SST_NVTX_RANGE();
    sst_status s = check_call(plan, x_dev, n, ws);
    if (s != SST_OK) return s;
    if (!V_dev || !Vd_dev) return fail(SST_EINVAL, "output pointer is NULL");
    SST_LAUNCHED_K(PK_STFT, (cudaStream_t)stream,
                   plan->kt->forward(plan->d, KIND_FWD_STFT, x_dev, ws_scalars(plan, ws), V_dev, Vd_dev,
                                     plan->grid_fwd_x, plan->smem_fwd_x, (cudaStream_t)stream),
                   "stft launch");
    return SST_OK;
}

SST_API sst_status sst_reassign_map(sst_plan_t plan, const float *x_dev, int64_t n, float *omega_dev,
                                    int32_t *dest_dev, void *ws, void *stream) {
    SST_NVTX_RANGE();
    sst_status s = check_call(plan, x_dev, n, ws);
    if (s != SST_OK) return s;
    if (!omega_dev || !dest_dev) return fail(SST_EINVAL, "output pointer is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (plan->d.relative) {
        s = run_prepass(plan, x_dev, ws_scalars(plan, ws), ws_partial(plan, ws), st, nullptr);
        if (s != SST_OK) return s;
    }
    SST_LAUNCHED_K(PK_MAP, st,
                   plan->kt->forward(plan->d, KIND_FWD_MAP, x_dev, ws_scalars(plan, ws), omega_dev, dest_dev,
                                     plan->grid_fwd_x, plan->smem_fwd_x, st),
                   "map launch");
    return SST_OK;
}

// ------------------------------------------------------------ second-order IF
// The forward with the second-order IF estimate (k_forward_so): the
// threshold's pre-pass as for sst_forward on a SST_TWO_PASS plan, then one
// launch of three packed FFTs per frame.
static sst_status run_forward_so(sst_plan_t pl, int kind, const float *x, void *out0, void *out1, void *ws,
                                 cudaStream_t st) {
    if (!pl->d.win2) return fail(SST_EUNSUPPORTED, "the second-order IF needs the built-in Gaussian window");
    const size_t smem = forward_so_smem_bytes(pl->kt->smem_frame, pl->d.nb, pl->d.nbo);
    int dev = 0;
    SST_CU(cudaGetDevice(&dev), "cudaGetDevice");
    int smax = 0;
    SST_CU(cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "device attributes");
    if (smem > (size_t)smax)
        return fail(SST_EUNSUPPORTED, "the second-order forward needs %zu bytes of shared memory (%d available)",
                    smem, smax);
    SST_CU(raise_smem(pl->kt, kind, smem), "cudaFuncSetAttribute");
    if (pl->d.relative || kind == KIND_FWD_SO_T) {
        sst_status s = run_prepass(pl, x, ws_scalars(pl, ws), ws_partial(pl, ws), st, nullptr);
        if (s != SST_OK) return s;
    }
    int occ = 1;
    if (pl->kt->occupancy(kind, smem, &occ) != cudaSuccess || occ < 1) occ = 1;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)occ * pl->num_sms * 2, pl->d.F));
    SST_LAUNCHED_K(kind == KIND_FWD_SO_T ? PK_FORWARD : PK_MAP, st,
                   pl->kt->forward(pl->d, kind, x, ws_scalars(pl, ws), out0, out1, grid, smem, st),
                   "second-order forward launch");
    return SST_OK;
}

SST_API sst_status sst_forward2(sst_plan_t plan, const float *x_dev, int64_t n, float *tfr_dev, void *ws,
                                void *stream) {
    SST_NVTX_RANGE();
    sst_status s = check_call(plan, x_dev, n, ws);
    if (s != SST_OK) return s;
    if (!tfr_dev) return fail(SST_EINVAL, "tfr pointer is NULL");
    return run_forward_so(plan, KIND_FWD_SO_T, x_dev, tfr_dev, nullptr, ws, (cudaStream_t)stream);
}

SST_API sst_status sst_reassign_map2(sst_plan_t plan, const float *x_dev, int64_t n, float *omega_dev,
                                     int32_t *dest_dev, void *ws, void *stream) {
    SST_NVTX_RANGE();
    sst_status s = check_call(plan, x_dev, n, ws);
    if (s != SST_OK) return s;
    if (!omega_dev || !dest_dev) return fail(SST_EINVAL, "output pointer is NULL");
    return run_forward_so(plan, KIND_FWD_SO_MAP, x_dev, omega_dev, dest_dev, ws, (cudaStream_t)stream);
}

SST_API sst_status sst_max_abs_v(sst_plan_t plan, const float *x_dev, int64_t n, float *maxv_dev, void *ws,
                                 void *stream) {
    SST_NVTX_RANGE();
    sst_status s = check_call(plan, x_dev, n, ws);
    if (s != SST_OK) return s;
    if (!maxv_dev) return fail(SST_EINVAL, "output pointer is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    SST_LAUNCHED_K(PK_ABSMAX, st,
                   plan->kt->absmax(plan->d, plan->absmax_cls, x_dev, ws_partial(plan, ws), plan->grid_absmax, plan->smem_absmax, st),
                   "absmax launch");
    SST_LAUNCHED_K(PK_GAMMA, st,
                   (k_gamma<<<1, 256, 0, st>>>(ws_partial(plan, ws), plan->grid_absmax, plan->gamma_frac2, 0, 1.f,
                                               plan->d.log2_nb, ws_scalars(plan, ws), maxv_dev, nullptr),
                    cudaGetLastError()),
                   "gamma launch");
    return SST_OK;
}

// ------------------------------------------------------------ split by frame ranges
// One signal over several GPUs (Sec. 2.1: frames are independent; Eq. 26's
// overlap-add couples neighbouring frames only): each part takes a contiguous
// range of inverse tiles and reads its frames' samples with an M-sample halo.
static sst_status part_check(sst_plan_t plan, const sst_part *part, const void *ws) {
    if (!plan || !part) return fail(SST_EINVAL, "plan or part is NULL");
    if (!ws) return fail(SST_EINVAL, "workspace is NULL");
    if (((uintptr_t)ws) & 255) return fail(SST_EINVAL, "workspace must be 256-byte aligned");
    const SstDev &d = plan->d;
    if (part->tile_begin < 0 || part->tile_end < part->tile_begin || part->tile_end > d.ntiles)
        return fail(SST_EINVAL, "tile range [%lld, %lld) outside [0, %lld)", (long long)part->tile_begin,
                    (long long)part->tile_end, (long long)d.ntiles);
    int dev = -1;
    SST_CU(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != plan->device) return fail(SST_EINVAL, "plan was created on device %d, current is %d", plan->device, dev);
    return SST_OK;
}

SST_API sst_status sst_part_layout(sst_plan_t plan, int32_t part, int32_t parts, sst_part *out) {
    if (!plan || !out) return fail(SST_EINVAL, "plan or out is NULL");
    if (parts < 1 || part < 0 || part >= parts) return fail(SST_EINVAL, "part %d of %d", part, parts);
    const SstDev &d = plan->d;
    sst_part r;
    memset(&r, 0, sizeof r);
    r.tile_begin = d.ntiles * part / parts;
    r.tile_end = d.ntiles * (part + 1) / parts;
    r.frame_begin = std::min<int64_t>(d.F, r.tile_begin * d.B);
    r.frame_end = std::min<int64_t>(d.F, r.tile_end * d.B);
    if (r.frame_end > r.frame_begin) {
        // the pre-pass packs frames in groups of four (k_absmax): a part reads
        // whole groups, so every frame's |S^g| comes out of the same packing
        // as in the unsplit pre-pass
        const int64_t q_lo = r.frame_begin / 4 * 4, q_hi = std::min<int64_t>(d.F, (r.frame_end + 3) / 4 * 4);
        r.x_begin = std::max<int64_t>(0, q_lo * d.hop - d.M);
        r.x_end = std::min<int64_t>(d.n, (q_hi - 1) * d.hop + d.M + 1);
    } else {
        r.x_begin = r.x_end = std::min<int64_t>(d.n, r.frame_begin * d.hop);
    }
    r.out_begin = part == 0 ? 0 : std::min<int64_t>(d.n, r.frame_begin * d.hop);
    r.out_end = part == parts - 1 ? d.n : std::min<int64_t>(d.n, r.frame_end * d.hop);
    // tiles whose overlap-add segments cover the part's output samples
    const int64_t BH = (int64_t)d.B * d.hop;
    if (r.out_end > r.out_begin) {
        const int64_t num = r.out_begin + d.M - d.seg_len + 1;
        r.need_begin = num <= 0 ? 0 : (num + BH - 1) / BH;
        r.need_end = std::min<int64_t>(d.ntiles, (r.out_end - 1 + d.M) / BH + 1);
    } else {
        r.need_begin = r.need_end = r.tile_begin;
    }
    *out = r;
    return SST_OK;
}

SST_API sst_status sst_part_segments(sst_plan_t plan, size_t *ola_offset, int32_t *seg_len, int64_t *tiles) {
    if (!plan) return fail(SST_EINVAL, "plan is NULL");
    if (ola_offset) *ola_offset = plan->ws_off_ola;
    if (seg_len) *seg_len = plan->d.seg_len;
    if (tiles) *tiles = plan->d.ntiles;
    return SST_OK;
}

SST_API sst_status sst_part_prepass(sst_plan_t plan, const sst_part *part, const float *x_dev, float *r_dev,
                                    void *ws, void *stream) {
    SST_NVTX_RANGE();
    sst_status s = part_check(plan, part, ws);
    if (s != SST_OK) return s;
    if (!r_dev) return fail(SST_EINVAL, "output pointer is NULL");
    if (!x_dev && part->x_end > part->x_begin) return fail(SST_EINVAL, "input pointer is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    float *partial = ws_partial(plan, ws);
    SstDev d = plan->d;
    d.xoff = part->x_begin;
    int count = 0;
    if (part->frame_end <= part->frame_begin) {
        SST_CU(cudaMemsetAsync(r_dev, 0, sizeof(float), st), "empty part");
        return SST_OK;
    }
    if (d.relative) {
        // whole groups of four frames (see sst_part_layout)
        d.frame_lo = part->frame_begin / 4 * 4;
        d.frame_hi = std::min<int64_t>(d.F, (part->frame_end + 3) / 4 * 4);
        const int64_t quads = (d.frame_hi + 3) / 4 - d.frame_lo / 4;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(plan->grid_absmax, quads));
        SST_LAUNCHED_K(PK_ABSMAX, st, plan->kt->absmax(d, plan->absmax_cls, x_dev, partial, grid, plan->smem_absmax, st),
                       "part pre-pass launch");
        count = grid;
    } else {
        const int64_t len = part->x_end - part->x_begin;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((len + 255) / 256, plan->grid_absmax));
        SST_LAUNCHED_K(PK_ABSMAX, st, launch_absx(x_dev, len, partial, grid, st), "part max |x| launch");
        count = grid;
    }
    SST_LAUNCHED_K(PK_GAMMA, st, (k_reduce_max<<<1, 256, 0, st>>>(partial, count, r_dev), cudaGetLastError()),
                   "part reduce launch");
    return SST_OK;
}

SST_API sst_status sst_part_forward_inverse(sst_plan_t plan, const sst_part *part, const float *x_dev,
                                            const float *r_dev, void *ws, void *stream) {
    SST_NVTX_RANGE();
    sst_status s = part_check(plan, part, ws);
    if (s != SST_OK) return s;
    if (!r_dev) return fail(SST_EINVAL, "pre-pass maximum pointer is NULL");
    if (!x_dev && part->x_end > part->x_begin) return fail(SST_EINVAL, "input pointer is NULL");
    if (!plan->fused_ok)
        return fail(SST_EUNSUPPORTED, "a split signal needs the fused kernel, whose %zu bytes of shared memory "
                    "this plan exceeds", plan->smem_fused);
    if (part->tile_end <= part->tile_begin) return SST_OK;
    cudaStream_t st = (cudaStream_t)stream;
    SstScalars *sc = ws_scalars(plan, ws);
    SST_LAUNCHED_K(PK_GAMMA, st,
                   launch_gamma(r_dev, 1, plan->gamma_frac2, plan->d.relative ? 0 : 1, plan->sum_abs_g,
                                plan->d.log2_nb, sc, nullptr, nullptr, st),
                   "part scalars launch");
    SstDev d = plan->d;
    d.xoff = part->x_begin;
    d.tile0 = part->tile_begin;
    d.ntiles = part->tile_end - part->tile_begin;   // the launch's grid
    SST_LAUNCHED_K(PK_FUSED, st, plan->kt->fused(d, plan->kind_fused, x_dev, sc, ws_ola(plan, ws), plan->smem_fused, st),
                   "part fused launch");
    return SST_OK;
}

SST_API sst_status sst_part_finalize(sst_plan_t plan, const sst_part *part, void *ws, float *xhat_dev,
                                     void *stream) {
    SST_NVTX_RANGE();
    sst_status s = part_check(plan, part, ws);
    if (s != SST_OK) return s;
    if (part->out_end < part->out_begin || part->out_begin < 0 || part->out_end > plan->d.n)
        return fail(SST_EINVAL, "output range outside the signal");
    if (part->out_end == part->out_begin) return SST_OK;
    if (!xhat_dev) return fail(SST_EINVAL, "xhat pointer is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t len = part->out_end - part->out_begin;
    const unsigned blocks = (unsigned)std::min<int64_t>((len + 255) / 256, 4096);
    SST_LAUNCHED_K(PK_FINALIZE, st,
                   (k_finalize_range<<<blocks, 256, 0, st>>>(plan->d, ws_ola(plan, ws), xhat_dev, part->out_begin,
                                                             part->out_end),
                    cudaGetLastError()),
                   "part finalize launch");
    return SST_OK;
}

// ------------------------------------------------------------ no-allocation forward
// Scratch for sst_forward_static: [0, 8) the call's SstScalars (threshold,
// fixed-point scale), [64 ...) one pre-pass maximum per CTA.  Host code must not use the symbol itself as an
// address (on the host it names a shadow variable); the device address is
// looked up once per device and cached.
static constexpr size_t kStaticFloats = SST_STATIC_SCRATCH_BYTES / sizeof(float);
static constexpr size_t kStaticHeader = 64;
static __device__ __align__(256) float g_static_scratch[kStaticFloats];
static std::mutex g_static_mu;
static float *g_static_addr[256];
static std::atomic<size_t> g_static_test_cap{0};   // test hook: a smaller capacity (0: the array's)

static sst_status static_scratch_address(int dev, float **out) {
    if (dev < 0 || dev >= 256) return fail(SST_EUNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch array");
        g_static_addr[dev] = (float *)p;
    }
    *out = g_static_addr[dev];
    return SST_OK;
}

SST_API sst_status sst_forward_static(sst_plan_t plan, const float *x_dev, int64_t n, float *tfr_dev,
                                      void *stream) {
    SST_NVTX_RANGE();
    if (!plan) return fail(SST_EINVAL, "plan is NULL");
    if (!x_dev || !tfr_dev) return fail(SST_EINVAL, "input or output pointer is NULL");
    if (n != plan->d.n)
        return fail(SST_EINVAL, "n = %lld differs from the plan's n = %lld", (long long)n, (long long)plan->d.n);
    const size_t need = kStaticHeader + (size_t)plan->grid_absmax;
    const size_t cap = g_static_test_cap.load() ? std::min(g_static_test_cap.load(), kStaticFloats) : kStaticFloats;
    if (need > cap)
        return fail(SST_EUNSUPPORTED, "this plan's pre-pass needs %zu scratch floats; the static array holds %zu",
                    need, cap);
    int dev = -1;
    SST_CU(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != plan->device) return fail(SST_EINVAL, "plan was created on device %d, current is %d", plan->device, dev);
    float *scratch = nullptr;
    sst_status s = static_scratch_address(dev, &scratch);
    if (s != SST_OK) return s;
    SstScalars *sc = (SstScalars *)scratch;
    float *partial = scratch + kStaticHeader;
    cudaStream_t st = (cudaStream_t)stream;
    s = run_prepass(plan, x_dev, sc, partial, st, nullptr, false);
    if (s != SST_OK) return s;
    SST_CU(plan->kt->forward(plan->d, plan->kind_fwd_t, x_dev, sc, tfr_dev, nullptr, plan->grid_fwd, plan->smem_fwd_t, st),
           "forward launch");
    count_launch();
    return SST_OK;
}

SST_API sst_status sst_test_static_capacity(size_t floats) {
    g_static_test_cap.store(floats);
    return SST_OK;
}

SST_API sst_status sst_check(sst_plan_t plan, const void *ws, void *stream) {
    SST_NVTX_RANGE();
    if (!plan || !ws) return fail(SST_EINVAL, "plan or workspace is NULL");
    SST_CU(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronise");
    unsigned w = 0;
    SST_CU(cudaMemcpy(&w, (const char *)ws + 192, sizeof w, cudaMemcpyDeviceToHost), "status read");
    if (w & SST_DEV_WAIT_EXPIRED)
        return fail(SST_ETIMEOUT, "a bounded wait for a staged copy (the forward's samples or the inverse's T rows) "
                    "gave up and the data were loaded directly instead%s",
                    (w & SST_DEV_COPY_LOST) ? "; the copy had not landed after a second bounded wait" : "");
    return SST_OK;
}

SST_API sst_status sst_test_withhold_sample_copy(sst_plan_t plan) {
    if (!plan) return fail(SST_EINVAL, "plan is NULL");
    plan->test_withhold_fwd.store(1);
    return SST_OK;
}

SST_API sst_status sst_test_withhold_row_copy(sst_plan_t plan) {
    if (!plan) return fail(SST_EINVAL, "plan is NULL");
    plan->test_withhold.store(1);
    return SST_OK;
}

SST_API sst_status sst_threshold_stats(sst_plan_t plan, const void *ws, int64_t *waiting, int64_t *bins,
                                       int32_t *fell_back) {
    if (!plan || !ws) return fail(SST_EINVAL, "plan or workspace is NULL");
    if (waiting) *waiting = 0;
    if (bins) *bins = 0;
    if (fell_back) *fell_back = 0;
    if (!plan->spec) return SST_OK;
    unsigned ctl[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    SST_CU(cudaDeviceSynchronize(), "device synchronise");
    SST_CU(cudaMemcpy(ctl, (const char *)ws + plan->ws_off_spec, sizeof ctl, cudaMemcpyDeviceToHost), "control read");
    if (waiting) *waiting = ctl[5];
    if (bins) *bins = ctl[6];
    if (fell_back) *fell_back = ctl[3] ? 1 : 0;
    return SST_OK;
}

// FP32 FMA throughput probe: eight independent fmaf chains per thread, full
// occupancy; the result is kept live by a store that never happens.
__global__ void __launch_bounds__(256) k_ffma_chains(float *__restrict__ out, int iters, float seed) {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = seed + (float)(threadIdx.x + j);
    const float m = 0.99999994f, c = 1.0e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], m, c);
    }
    float t = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) t += a[j];
    if (t == 12345.678f) out[0] = t;
}

SST_API sst_status sst_fp32_peak(double *tflops, void *stream) {
    if (!tflops) return fail(SST_EINVAL, "output pointer is NULL");
    int dev = 0, sms = 0;
    SST_CU(cudaGetDevice(&dev), "cudaGetDevice");
    SST_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attributes");
    cudaStream_t st = (cudaStream_t)stream;
    float *out = nullptr;
    SST_CU(cudaMalloc(&out, 256), "probe buffer");
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    const int blocks = sms * 8, iters = 16384;
    float ms = 0.f;
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {   // the last of three launches is timed
        e = cudaEventRecord(a, st);
        if (e == cudaSuccess) {
            k_ffma_chains<<<blocks, 256, 0, st>>>(out, iters, 1.0f + r);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        count_launch();
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess) return cuda_fail(e, "FP32 probe");
    *tflops = 2.0 * 8.0 * iters * (double)blocks * 256.0 / (ms * 1e-3) / 1e12;
    return SST_OK;
}

SST_API sst_status sst_sync(void *stream) {
    SST_NVTX_RANGE();
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronise");
    return SST_OK;
}

SST_API uint64_t sst_launch_count(void) { return sst::g_launches.load(); }

SST_API sst_status sst_profile_enable(int on) {
    g_prof_on.store(on ? 1 : 0);
    return SST_OK;
}

SST_API sst_status sst_profile_collect(double *ms, uint64_t *counts) {
    std::vector<ProfRec> recs;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        recs.swap(g_prof);
    }
    if (ms) for (int i = 0; i < SST_PROFILE_KINDS; ++i) ms[i] = 0.0;
    if (counts) for (int i = 0; i < SST_PROFILE_KINDS; ++i) counts[i] = 0;
    sst_status st = SST_OK;
    for (auto &r : recs) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess && st == SST_OK) st = cuda_fail(e, "profile event");
        if (ms) ms[r.kind] += t;
        if (counts) counts[r.kind] += 1;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    return st;
}

SST_API const char *sst_profile_kind_name(int kind) {
    if (kind < 0 || kind >= SST_PROFILE_KINDS) return "";
    return kPkNames[kind];
}

SST_API const char *sst_status_string(sst_status s) {
    switch (s) {
        case SST_OK: return "SST_OK";
        case SST_EINVAL: return "SST_EINVAL";
        case SST_ENOMEM: return "SST_ENOMEM";
        case SST_ECUDA: return "SST_ECUDA";
        case SST_EBUSY: return "SST_EBUSY";
        case SST_ETIMEOUT: return "SST_ETIMEOUT";
        case SST_EUNSUPPORTED: return "SST_EUNSUPPORTED";
        case SST_EINTERNAL: return "SST_EINTERNAL";
    }
    return "SST_<unknown>";
}

SST_API const char *sst_last_error(void) { return g_err.c_str(); }
